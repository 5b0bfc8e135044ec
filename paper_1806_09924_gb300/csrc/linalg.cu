// Deterministic reductions, scans and sparse kernels shared by the AMG and the
// Krylov solver.  Every reduction uses a fixed grid and a fixed combination
// order, so a result depends only on the input size, never on timing.
#include <algorithm>

#include "pff_internal.h"

namespace pff {

namespace {

constexpr int RB = 256;   // reduction block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// block sum of one value per thread -> returned in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    r = warp_max(r);
  }
  __syncthreads();
  return r;
}

int red_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(RED_PARTIALS, (n + RB - 1) / RB)); }

__global__ void k_dot(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                      double* __restrict__ part) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a += x[i] * y[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// FP32 vectors: products summed in FP32 per thread, blocks and partials in FP64
__global__ void k_dot_f32(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
                          double* __restrict__ part) {
  __shared__ double sh[32];
  float a = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a += x[i] * y[i];
  const double s = block_sum((double)a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_nrm_inf(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a = fmax(a, fabs(x[i]));
  a = block_max(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void k_final(const double* __restrict__ part, int np, int stride, int is_max,
                        double* __restrict__ out) {
  __shared__ double sh[32];
  const double* p = part + (int64_t)blockIdx.x * stride;
  double a = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) a = is_max ? fmax(a, p[k]) : a + p[k];
  a = is_max ? block_max(a, sh) : block_sum(a, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

// up to 8 dot products per pass: out_k = <V_k, w>
template <int K>
__global__ void k_multidot(const double* __restrict__ V, int64_t ld, int k0,
                           const double* __restrict__ w, int64_t n, double* __restrict__ part,
                           int pstride) {
  __shared__ double sh[32];
  double a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] += V[(int64_t)(k0 + k) * ld + i] * wi;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double s = block_sum(a[k], sh);
    if (threadIdx.x == 0) part[(int64_t)(k0 + k) * pstride + blockIdx.x] = s;
  }
}

__global__ void k_multi_axpy(const double* __restrict__ V, int64_t ld, int nv,
                             const double* __restrict__ h, double* __restrict__ w, int64_t n,
                             double sign) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int k = 0; k < nv; ++k) a += h[k] * V[(int64_t)k * ld + i];
  w[i] += sign * a;
}

// ------------------------------------------------ Gram-Schmidt (mixed) ---
// GB300 executes FP64 arithmetic at a small fraction of its FP32 rate, which
// puts an FP64 multiply-add per streamed double below the HBM roofline.  The
// mixed-precision Krylov path therefore takes its projection coefficients and
// norms in FP32: from FP32 views of the FP64 data (f32_view: the high word
// re-biased with integer operations).  The view of each basis vector is stored
// when the vector is normalised, so the coefficient pass streams 4 bytes per
// element of V instead of 8.  FP64 arithmetic is kept only for the update w <- w - V h,
// whose coefficients h are the ones stored in the Hessenberg matrix, so the
// Arnoldi relation holds to FP64 rounding.

template <int K>
__device__ __forceinline__ void block_sum_f(float (&v)[K], float (*sh)[K]) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < K; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    if (l == 0) sh[w][c] = v[c];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    float r = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i][threadIdx.x];
    v[0] = r;   // thread c holds the block sum of value c
  }
  __syncthreads();
}

constexpr int GS_CH = 8;

// block b owns rows [b R, b R + R): it stages the FP32 view of w there in shared
// memory, then sweeps the FP32 basis vectors GS_CH at a time.
// part[k g + b] = block partial of <Vf_k, w> (k < nv); part[nv g + b] = of ||w||^2
__global__ void __launch_bounds__(RB) k_gs_dot(const float* __restrict__ Vf, int64_t ld, int nv,
                                                const double* __restrict__ w, int64_t n, int R,
                                                float* __restrict__ part) {
  extern __shared__ float swf[];
  __shared__ float red[RB / 32][GS_CH];
  const int g = gridDim.x, b = blockIdx.x;
  const int64_t r0 = (int64_t)b * R;
  const int len = (int)std::max<int64_t>(0, std::min<int64_t>(R, n - r0));
  float nrm[GS_CH] = {};
  for (int i = threadIdx.x; i < len; i += RB) {
    const float f = f32_view(w[r0 + i]);
    swf[i] = f;
    nrm[0] += f * f;
  }
  block_sum_f<GS_CH>(nrm, red);   // also orders the shared-memory stores before the reads
  if (threadIdx.x == 0) part[(int64_t)nv * g + b] = nrm[0];
  for (int k0 = 0; k0 < nv; k0 += GS_CH) {
    float acc[GS_CH] = {};
    const float* Vk = Vf + (int64_t)k0 * ld + r0;
    const int kc = min(GS_CH, nv - k0);
    for (int i = threadIdx.x; i < len; i += RB) {
      const float wf = swf[i];
#pragma unroll
      for (int c = 0; c < GS_CH; ++c)
        if (c < kc) acc[c] += Vk[(int64_t)c * ld + i] * wf;
    }
    block_sum_f<GS_CH>(acc, red);
    if (threadIdx.x < kc) part[(int64_t)(k0 + threadIdx.x) * g + b] = acc[0];
  }
}

// w <- w - sum_k h_k V_k in FP64; part[b] = block partial of ||w_new||^2 (FP32 view)
__global__ void __launch_bounds__(RB) k_gs_axpy(const double* __restrict__ V, int64_t ld, int nv,
                                                 const double* __restrict__ h, double* __restrict__ w,
                                                 int64_t n, float* __restrict__ part) {
  __shared__ double sh[64];
  __shared__ float red[RB / 32][1];
  if (threadIdx.x < nv) sh[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  float nrm[1] = {0.f};
  for (int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    double a = w[i];
    int k = 0;
    for (; k + 4 <= nv; k += 4) {
      const double v0 = V[(int64_t)k * ld + i], v1 = V[(int64_t)(k + 1) * ld + i];
      const double v2 = V[(int64_t)(k + 2) * ld + i], v3 = V[(int64_t)(k + 3) * ld + i];
      a = fma(-sh[k], v0, a);
      a = fma(-sh[k + 1], v1, a);
      a = fma(-sh[k + 2], v2, a);
      a = fma(-sh[k + 3], v3, a);
    }
    for (; k < nv; ++k) a = fma(-sh[k], V[(int64_t)k * ld + i], a);
    w[i] = a;
    const float f = f32_view(a);
    nrm[0] += f * f;
  }
  block_sum_f<1>(nrm, red);
  if (threadIdx.x == 0) part[blockIdx.x] = nrm[0];
}

// out[b] = sum of the g FP32 partials of row b, accumulated in FP64
__global__ void k_gs_final(const float* __restrict__ part, int g, double* __restrict__ out) {
  __shared__ double sh[32];
  const float* p = part + (int64_t)blockIdx.x * g;
  double a = 0.0;
  for (int k = threadIdx.x; k < g; k += blockDim.x) a += (double)p[k];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

// -------------------------------------------------------------------- scan --
constexpr int SB = 1024;

__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, int n,
                             int* __restrict__ bsum) {
  __shared__ int sh[SB];
  const int i = blockIdx.x * SB + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < SB; o <<= 1) {
    int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;   // exclusive
  if (threadIdx.x == SB - 1) bsum[blockIdx.x] = sh[SB - 1];
}

__global__ void k_scan_sums(int* __restrict__ bsum, int nb, int* __restrict__ total) {
  if (threadIdx.x != 0) return;
  int run = 0;
  for (int b = 0; b < nb; ++b) {
    const int v = bsum[b];
    bsum[b] = run;
    run += v;
  }
  *total = run;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ bsum,
                           const int* __restrict__ total) {
  const int i = blockIdx.x * SB + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
  if (i == 0) out[n] = *total;
}

}  // namespace

void dot_dev(const double* x, const double* y, int64_t n, double* out, double* partials,
             cudaStream_t s) {
  const int g = red_grid(n);
  ProfScope ps("dot", (x == y ? 8.0 : 16.0) * n, s, 2);
  k_dot<<<g, RB, 0, s>>>(x, y, n, partials);
  k_final<<<1, RB, 0, s>>>(partials, g, 0, 0, out);
  PFF_LAUNCH("dot");
}

void dot_dev_f32(const float* x, const float* y, int64_t n, double* out, double* partials,
                 cudaStream_t s) {
  const int g = red_grid(n);
  ProfScope ps("dot_f32", (x == y ? 4.0 : 8.0) * n, s, 2);
  k_dot_f32<<<g, RB, 0, s>>>(x, y, n, partials);
  k_final<<<1, RB, 0, s>>>(partials, g, 0, 0, out);
  PFF_LAUNCH("dot_f32");
}

void nrm_inf_dev(const double* x, int64_t n, double* out, double* partials, cudaStream_t s) {
  const int g = red_grid(n);
  ProfScope ps("nrm_inf", 8.0 * n, s, 2);
  k_nrm_inf<<<g, RB, 0, s>>>(x, n, partials);
  k_final<<<1, RB, 0, s>>>(partials, g, 0, 1, out);
  PFF_LAUNCH("nrm_inf");
}

void multidot_dev(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* out,
                  double* partials, cudaStream_t s) {
  // up to 1024 blocks (about 7 per SM): enough loads in flight to stream V at HBM speed;
  // the partial sums need nv * g <= 65536 doubles (nv <= 64)
  const int g = red_grid(n);
  ProfScope ps("multidot", 8.0 * n * (nv + 1.0), s, (nv + 7) / 8 + 1);
  int k0 = 0;
  while (k0 < nv) {
    const int k = std::min(8, nv - k0);
    switch (k) {
      case 8: k_multidot<8><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
      case 7: k_multidot<7><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
      case 6: k_multidot<6><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
      case 5: k_multidot<5><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
      case 4: k_multidot<4><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
      case 3: k_multidot<3><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
      case 2: k_multidot<2><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
      default: k_multidot<1><<<g, RB, 0, s>>>(V, ld, k0, w, n, partials, g); break;
    }
    k0 += k;
  }
  k_final<<<nv, RB, 0, s>>>(partials, g, g, 0, out);
  PFF_LAUNCH("multidot");
}

void multi_axpy_dev(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n,
                    double sign, cudaStream_t s) {
  ProfScope ps("multi_axpy", 8.0 * n * (nv + 2.0), s);
  k_multi_axpy<<<grid_for(n, 256), 256, 0, s>>>(V, ld, nv, h, w, n, sign);
  PFF_LAUNCH("multi_axpy");
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 132;
  }
  return n;
}

int64_t l2_cache_bytes() {
  static const int64_t l2 = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    return (int64_t)v;
  }();
  return l2;
}

// resident blocks per SM of a kernel (registers and shared memory permitting)
template <class K>
int resident_blocks(K kernel, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, RB, smem) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 4;
  }
  return b;
}

int gs_grid(int64_t n, int* rows_per_block) {
  // one full wave (every SM holding as many blocks as fit), more blocks when a
  // block's rows would overflow the staging buffer (GS_MAX_ROWS floats)
  static int waves_blocks = 0;
  if (waves_blocks == 0)
    waves_blocks = sm_count() * resident_blocks(k_gs_dot, sizeof(float) * (GS_MAX_ROWS / 2));
  int64_t g = std::max<int64_t>(waves_blocks, (n + GS_MAX_ROWS - 1) / GS_MAX_ROWS);
  g = std::max<int64_t>(1, std::min<int64_t>(g, n));
  *rows_per_block = (int)((n + g - 1) / g);
  return (int)((n + *rows_per_block - 1) / *rows_per_block);
}

void gs_dot_dev(const float* Vf, int64_t ld, int nv, const double* w, int64_t n, float* part,
                double* out, cudaStream_t s) {
  int R = 0;
  const int g = gs_grid(n, &R);
  if (R > GS_MAX_ROWS || g > GS_MAX_BLOCKS || nv > 64)
    fail(PFF_ERR_INVALID_ARG, "mixed Gram-Schmidt: system or basis too large");
  ProfScope ps("gs_dot", n * (4.0 * nv + 8.0), s, 2);
  k_gs_dot<<<g, RB, sizeof(float) * R, s>>>(Vf, ld, nv, w, n, R, part);
  k_gs_final<<<nv + 1, RB, 0, s>>>(part, g, out);
  PFF_LAUNCH("gs_dot");
}

void gs_axpy_dev(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n,
                 float* part, double* nrm2, cudaStream_t s) {
  if (nv > 64) fail(PFF_ERR_INVALID_ARG, "mixed Gram-Schmidt: basis too large");
  static int wave = 0;
  if (wave == 0) wave = sm_count() * resident_blocks(k_gs_axpy, 0);
  const int g = (int)std::min<int64_t>(wave, std::max<int64_t>(1, (n + RB - 1) / RB));
  ProfScope ps("gs_axpy", 8.0 * n * (nv + 2.0), s, 2);
  k_gs_axpy<<<g, RB, 0, s>>>(V, ld, nv, h, w, n, part);
  k_gs_final<<<1, RB, 0, s>>>(part, g, nrm2);
  PFF_LAUNCH("gs_axpy");
}

void exclusive_scan_int(const int* in, int* out, int n, int* total_host, cudaStream_t s) {
  const int nb = std::max(1, (n + SB - 1) / SB);
  int* bsum = dalloc<int>(nb + 1);
  int* tot = bsum + nb;
  count_launch(3);
  k_scan_block<<<nb, SB, 0, s>>>(in, out, n, bsum);
  k_scan_sums<<<1, 32, 0, s>>>(bsum, nb, tot);
  k_scan_add<<<nb, SB, 0, s>>>(out, n, bsum, tot);
  PFF_LAUNCH("scan");
  if (total_host) {
    PFF_CUDA(cudaMemcpyAsync(total_host, tot, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFF_CUDA(cudaStreamSynchronize(s));
  }
  PFF_CUDA(cudaStreamSynchronize(s));
  dfree(bsum);
}

void Bsr::release() {
  dfree(rowptr);
  dfree(col);
  dfree(val);
  dfree(valf);
  dfree(sell_off);
  dfree(sell_col);
  dfree(sell_valf);
  sell_off = sell_col = nullptr;
  sell_valf = nullptr;
  rowptr = nullptr;
  col = nullptr;
  val = nullptr;
  valf = nullptr;
  nrows = ncols = 0;
  nnzb = 0;
}

}  // namespace pff
