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
  rowptr = nullptr;
  col = nullptr;
  val = nullptr;
  valf = nullptr;
  nrows = ncols = 0;
  nnzb = 0;
}

}  // namespace pff
