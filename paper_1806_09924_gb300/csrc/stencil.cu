// Level-0 smoother of both AMG hierarchies: Chebyshev steps and residuals on
// the assembled node stencils (Kuu with block size d, Kpp with block size 1,
// slot-major as produced by the element kernels), in FP32 or FP64, plus the
// node-major FP32 copy of the 2d displacement stencil and the inverse
// diagonals.  These are the bandwidth-bound kernels of every V-cycle (Section
// 3.1: block-diagonal AMG preconditioner), kept in a file of their own.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>

#include "pff_internal.h"

namespace pff {

namespace {

// ------------------------------------------- stencil smoother (AMG level 0) --
// The finest AMG level of each block is the assembled node stencil itself
// (Kuu with B = d, Kpp with B = 1, slot-major).  acc = K x over the 3^D
// neighbours of node i, without branches: a neighbour outside the mesh is
// replaced by node i itself and its product selected away, so every load is
// in bounds and independent of the others, and all of them can be in flight
// together (node indices fit in 32 bits).
//
// The stencils are symmetric (M_uu and the reduced M_phi_phi: Dirichlet and
// active rows and columns are eliminated alike), so the FP32 copies keep only
// the centre slot and the slots after it (h = s - C, C = (3^D - 1) / 2).  The
// block of a slot s < C is the transpose of the block node j = i + offset(s)
// stores for the opposite slot 3^D - 1 - s, read from j's column: consecutive
// threads still read consecutive addresses, and the copy moves 5/9 (2d) or
// 14/27 (3d) of the full stencil's bytes.  FP64 stencils are full.
//
// SK (stream K): stencil loads marked evict-first (ld.global.cs).  When the
// stored stencil is about the size of L2, this keeps the gathered vectors
// cached instead of the stencil, which is read once per step anyway.
template <bool SK, class T>
__device__ __forceinline__ T ld_stencil(const T* p) {
  if constexpr (SK) return __ldcs(p);
  else return *p;
}

// Explicitly rounded arithmetic (no contraction left to the compiler): the
// kernel variants of one step then produce bit-identical results.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// One Chebyshev update of component r: res = dinv (b - acc), d = cd d + cr res,
// x_out = x_in + d (zero start: d = cr res, x_out = d).
template <class T>
__device__ __forceinline__ void cheb_update(int64_t r, T acc, const T* __restrict__ dinv,
                                            const T* __restrict__ rhs, const T* __restrict__ xin,
                                            T* __restrict__ xout, T* __restrict__ d, T cd, T cr,
                                            int zero_x, const double* __restrict__ rhs64,
                                            T* __restrict__ rhs_store, double* __restrict__ out64) {
  T bv;
  if (rhs64) {
    bv = (T)rhs64[r];
    rhs_store[r] = bv;
  } else {
    bv = rhs[r];
  }
  const T res = rn_mul(dinv[r], rn_sub(bv, acc));
  const T crr = rn_mul(cr, res);
  const T dn = zero_x ? crr : rn_fma(cd, d[r], crr);
  const T xo = zero_x ? dn : rn_add(xin[r], dn);
  if (out64) {
    out64[r] = (double)xo;
  } else {
    d[r] = dn;
    xout[r] = xo;
  }
}

template <class T, int D, int B, bool SK>
__device__ __forceinline__ void stencil_apply(const MeshDev& m, int64_t n, int i,
                                              const T* __restrict__ K, const T* __restrict__ x,
                                              T (&acc)[B]) {
  constexpr int NS = D == 2 ? 9 : 27;
  constexpr int C = NS / 2;
  constexpr bool HALF = sizeof(T) == 4;
  const int n0 = m.nn[0], n1 = m.nn[1];
  const int ix = i % n0;
  const int r = i / n0;
  const int iy = D == 2 ? r : r % n1;
  const int iz = D == 2 ? 0 : r / n1;
  const bool lo[3] = {ix > 0, iy > 0, iz > 0};
  const bool hi[3] = {ix < n0 - 1, iy < n1 - 1, D == 3 && iz < m.nn[2] - 1};
#pragma unroll
  for (int a = 0; a < B; ++a) acc[a] = T(0);
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = D == 3 ? s / 9 - 1 : 0;
    const bool ok = (ox < 0 ? lo[0] : ox > 0 ? hi[0] : true) &&
                    (oy < 0 ? lo[1] : oy > 0 ? hi[1] : true) &&
                    (oz < 0 ? lo[2] : oz > 0 ? hi[2] : true);
    const int j = ok ? i + ox + oy * n0 + oz * n0 * n1 : i;
    T xj[B];
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const T v = x[(int64_t)j * B + c];
      xj[c] = ok ? v : T(0);
    }
#pragma unroll
    for (int a = 0; a < B; ++a)
#pragma unroll
      for (int c = 0; c < B; ++c) {
        T k;
        if (!HALF) k = ld_stencil<SK>(K + ((int64_t)(s * B + a) * B + c) * n + i);
        else if (s >= C) k = ld_stencil<SK>(K + ((int64_t)((s - C) * B + a) * B + c) * n + i);
        else k = ld_stencil<SK>(K + ((int64_t)((NS - 1 - s - C) * B + c) * B + a) * n + j);
        acc[a] = rn_fma(ok ? k : T(0), xj[c], acc[a]);
      }
  }
}

// Launch shape per instantiation.  With __launch_bounds__(256) alone the compiler
// packs the 3d displacement step into 32 registers and serialises its 27 x 9
// stencil loads (2.0 TB/s on the 128^3 mesh, measured); capping it at 128
// registers with 4 blocks of 128 threads per SM keeps every load of a node in
// flight (4.5 TB/s, bit-identical results).  The phase-field steps (B = 1) run
// best with 6 blocks of 256 threads per SM (2.5 -> 3.7 TB/s).
template <int D, int B>
struct StencilShape {
  static constexpr int threads = (D == 3 && B == 3) ? 128 : 256;
  static constexpr int min_blocks = B == 1 ? 6 : 4;
};

// One Chebyshev step fused with the operator apply:
// res = dinv .* (rhs - K x_in),  d = cd d + cr res,  x_out = x_in + d.
// With zero_x the iterate starts at 0 (no apply).  The first step of a mixed
// V-cycle takes the FP64 right-hand side (rhs64, also stored as T into
// rhs_store for the later steps) and the last one writes the FP64 result
// (out64, instead of x_out and d), which saves two conversion passes.
template <class T, int D, int B, bool SK>
__global__ void __launch_bounds__(StencilShape<D, B>::threads, StencilShape<D, B>::min_blocks)
    k_stencil_cheb(MeshDev m, int64_t n,
                                                      const T* __restrict__ K,
                                                      const T* __restrict__ dinv,
                                                      const T* __restrict__ rhs,
                                                      const T* __restrict__ xin,
                                                      T* __restrict__ xout, T* __restrict__ d,
                                                      T cd, T cr, int zero_x,
                                                      const double* __restrict__ rhs64,
                                                      T* __restrict__ rhs_store,
                                                      double* __restrict__ out64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T acc[B];
  if (zero_x) {
#pragma unroll
    for (int a = 0; a < B; ++a) acc[a] = T(0);
  } else {
    stencil_apply<T, D, B, SK>(m, n, i, K, xin, acc);
  }
#pragma unroll
  for (int a = 0; a < B; ++a)
    cheb_update<T>((int64_t)i * B + a, acc[a], dinv, rhs, xin, xout, d, cd, cr, zero_x, rhs64,
                   rhs_store, out64);
}

// 2d displacement block in FP32 with the node-major layout Kq[(h n + i) * 4 + 2a + c]
// (slots s = h + 4 >= 4 only, as above): each node's 2x2 block of a slot is one
// 16-byte load, each neighbour's x one 8-byte load.  RESID: r = rhs - K x;
// otherwise one Chebyshev step as above.
template <bool RESID, bool SK>
__device__ __forceinline__ void stencil_q2(const MeshDev& m, int n, const float* __restrict__ Kq,
                                           const float* __restrict__ dinv,
                                           const float* __restrict__ rhs,
                                           const float* __restrict__ xin, float* __restrict__ out,
                                           float* __restrict__ d, float cd, float cr, int zero_x,
                                           const double* __restrict__ rhs64,
                                           float* __restrict__ rhs_store,
                                           double* __restrict__ out64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a0 = 0.f, a1 = 0.f;
  if (RESID || !zero_x) {
    const int n0 = m.nn[0];
    const int ix = i % n0, iy = i / n0;
    const bool lx = ix > 0, hx = ix < n0 - 1, ly = iy > 0, hy = iy < m.nn[1] - 1;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      const int ox = s % 3 - 1, oy = s / 3 - 1;
      const bool ok = (ox < 0 ? lx : ox > 0 ? hx : true) && (oy < 0 ? ly : oy > 0 ? hy : true);
      const int j = ok ? i + ox + oy * n0 : i;
      const float2 x = reinterpret_cast<const float2*>(xin)[j];
      float4 k;
      if (s >= 4) {
        k = ld_stencil<SK>(reinterpret_cast<const float4*>(Kq) + (int64_t)(s - 4) * n + i);
      } else {
        const float4 kt = ld_stencil<SK>(reinterpret_cast<const float4*>(Kq) + (int64_t)(4 - s) * n + j);
        k = make_float4(kt.x, kt.z, kt.y, kt.w);   // transpose of node j's block
      }
      const float x0 = ok ? x.x : 0.f, x1 = ok ? x.y : 0.f;
      a0 += k.x * x0 + k.y * x1;
      a1 += k.z * x0 + k.w * x1;
    }
  }
  float2 b;
  if (!RESID && rhs64) {
    // scalar FP64 accesses: an FP64 vector may start at an odd element offset
    b = make_float2((float)rhs64[2 * (int64_t)i], (float)rhs64[2 * (int64_t)i + 1]);
    reinterpret_cast<float2*>(rhs_store)[i] = b;
  } else {
    b = reinterpret_cast<const float2*>(rhs)[i];
  }
  if constexpr (RESID) {
    reinterpret_cast<float2*>(out)[i] = make_float2(b.x - a0, b.y - a1);
  } else {
    const float2 di = reinterpret_cast<const float2*>(dinv)[i];
    float2 dn = make_float2(cr * di.x * (b.x - a0), cr * di.y * (b.y - a1));
    float2 xo = dn;
    if (!zero_x) {
      const float2 dd = reinterpret_cast<const float2*>(d)[i];
      const float2 xi = reinterpret_cast<const float2*>(xin)[i];
      dn.x += cd * dd.x;
      dn.y += cd * dd.y;
      xo = make_float2(xi.x + dn.x, xi.y + dn.y);
    }
    if (out64) {
      out64[2 * (int64_t)i] = (double)xo.x;
      out64[2 * (int64_t)i + 1] = (double)xo.y;
    } else {
      reinterpret_cast<float2*>(d)[i] = dn;
      reinterpret_cast<float2*>(out)[i] = xo;
    }
  }
}

// 128-thread blocks with a minimum of one block per SM: the compiler then keeps
// all nine neighbour loads in flight (about 70 registers); with 256-thread blocks
// it packs the kernel into 32 registers and serialises them (20-25 % slower on
// a 1024^2 mesh, measured)
constexpr int Q2_BLK = 128;

template <bool SK>
__global__ void __launch_bounds__(Q2_BLK, 1) k_stencil_cheb_q2(MeshDev m, int n, const float* __restrict__ Kq,
                                                         const float* __restrict__ dinv,
                                                         const float* __restrict__ rhs,
                                                         const float* __restrict__ xin,
                                                         float* __restrict__ xout,
                                                         float* __restrict__ d, float cd, float cr,
                                                         int zero_x,
                                                         const double* __restrict__ rhs64,
                                                         float* __restrict__ rhs_store,
                                                         double* __restrict__ out64) {
  stencil_q2<false, SK>(m, n, Kq, dinv, rhs, xin, xout, d, cd, cr, zero_x, rhs64, rhs_store, out64);
}

template <bool SK>
__global__ void __launch_bounds__(Q2_BLK, 1) k_stencil_resid_q2(MeshDev m, int n,
                                                          const float* __restrict__ Kq,
                                                          const float* __restrict__ rhs,
                                                          const float* __restrict__ x,
                                                          float* __restrict__ r) {
  stencil_q2<true, SK>(m, n, Kq, nullptr, rhs, x, r, nullptr, 0.f, 0.f, 0, nullptr, nullptr, nullptr);
}

// node-major FP32 copy of the 2d displacement stencil, slots 4..8 (2 x 2 blocks)
__global__ void k_stencil_to_q2(int64_t n, const double* __restrict__ K, float* __restrict__ Kq) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * n) return;
  const int64_t h = t / n, i = t - h * n, s = h + 4;
  float4 q;
  q.x = (float)K[(s * 4 + 0) * n + i];
  q.y = (float)K[(s * 4 + 1) * n + i];
  q.z = (float)K[(s * 4 + 2) * n + i];
  q.w = (float)K[(s * 4 + 3) * n + i];
  reinterpret_cast<float4*>(Kq)[t] = q;
}

// r = rhs - K x
template <class T, int D, int B, bool SK>
__global__ void __launch_bounds__(StencilShape<D, B>::threads, StencilShape<D, B>::min_blocks)
    k_stencil_resid(MeshDev m, int64_t n,
                                                       const T* __restrict__ K,
                                                       const T* __restrict__ rhs,
                                                       const T* __restrict__ x,
                                                       T* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T acc[B];
  stencil_apply<T, D, B, SK>(m, n, i, K, x, acc);
#pragma unroll
  for (int a = 0; a < B; ++a) r[(int64_t)i * B + a] = rn_sub(rhs[(int64_t)i * B + a], acc[a]);
}

// 3d displacement block in FP32, one output component per warp ("rows"): the
// three warps of a group of 32 nodes compute rows a = 0, 1, 2 of the same 32
// nodes.  Each thread then carries one accumulator and 27 x 3 stencil loads
// instead of 3 accumulators and 27 x 9 loads, so four times as many threads
// fit in the register file and more loads are in flight per SM; the three
// warps read the same x values (from L1).  Every row accumulates its products
// in the same order as the node-per-thread kernel, so both give bit-identical
// results.  RESID: out = rhs - K x; otherwise one Chebyshev step.
constexpr int ROWS_GROUPS = 4;                 // groups of 32 nodes per block
constexpr int ROWS_THREADS = 96 * ROWS_GROUPS;

template <bool RESID, bool SK, int MINB>
__global__ void __launch_bounds__(ROWS_THREADS, MINB)
    k_stencil_rows3(MeshDev m, int n, const float* __restrict__ K, const float* __restrict__ dinv,
                    const float* __restrict__ rhs, const float* __restrict__ xin,
                    float* __restrict__ out, float* __restrict__ d, float cd, float cr, int zero_x,
                    const double* __restrict__ rhs64, float* __restrict__ rhs_store,
                    double* __restrict__ out64) {
  constexpr int NS = 27, C = 13, B = 3;
  const int w = threadIdx.x >> 5;
  const int a = w % 3;
  const int i = (blockIdx.x * ROWS_GROUPS + w / 3) * 32 + (threadIdx.x & 31);
  if (i >= n) return;
  float acc = 0.f;
  if (RESID || !zero_x) {
    const int n0 = m.nn[0], n1 = m.nn[1];
    const int ix = i % n0;
    const int r = i / n0;
    const int iy = r % n1, iz = r / n1;
    const bool lo[3] = {ix > 0, iy > 0, iz > 0};
    const bool hi[3] = {ix < n0 - 1, iy < n1 - 1, iz < m.nn[2] - 1};
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = s / 9 - 1;
      const bool ok = (ox < 0 ? lo[0] : ox > 0 ? hi[0] : true) &&
                      (oy < 0 ? lo[1] : oy > 0 ? hi[1] : true) &&
                      (oz < 0 ? lo[2] : oz > 0 ? hi[2] : true);
      const int j = ok ? i + ox + oy * n0 + oz * n0 * n1 : i;
      float xj[B];
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const float v = xin[(int64_t)j * B + c];
        xj[c] = ok ? v : 0.f;
      }
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float k;
        if (s >= C) k = ld_stencil<SK>(K + ((int64_t)((s - C) * B + a) * B + c) * n + i);
        else k = ld_stencil<SK>(K + ((int64_t)((NS - 1 - s - C) * B + c) * B + a) * n + j);
        acc = rn_fma(ok ? k : 0.f, xj[c], acc);
      }
    }
  }
  const int64_t r = (int64_t)i * B + a;
  if (RESID) {
    out[r] = rn_sub(rhs[r], acc);
    return;
  }
  cheb_update<float>(r, acc, dinv, rhs, xin, out, d, cd, cr, zero_x, rhs64, rhs_store, out64);
}

// inverse diagonal of a node stencil (block size B, centre slot c0)
__global__ void k_stencil_dinv(int64_t n, int B, int c0, const double* __restrict__ K,
                               double* __restrict__ dinv, float* __restrict__ dinvf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = 0; a < B; ++a) {
    const double v = K[((int64_t)(c0 * B + a) * B + a) * n + i];
    const double r = v != 0.0 ? 1.0 / v : 0.0;
    dinv[i * B + a] = r;
    if (dinvf) dinvf[i * B + a] = (float)r;
  }
}

}  // namespace

namespace {
inline double NSd(int d) { return d == 2 ? 9.0 : 27.0; }
// slots a stencil copy of element size es holds (FP32 copies: centre and after)
inline double slots_stored(int d, size_t es) { return es == 4 ? (NSd(d) + 1.0) / 2.0 : NSd(d); }
// whether the stored stencil of n nodes (block size b, element size es) fits in L2:
// then its loads are marked evict-first (measured: 25 % faster for the 2d
// displacement step at 1024^2, neutral on smaller stencils, 4 % slower on one
// 2.7 times the L2)
bool stream_stencil(int d, int b, size_t es, int64_t n) {
  return slots_stored(d, es) * b * b * es * (double)n <= (double)l2_cache_bytes();
}
}  // namespace

namespace {
// Kernel variant of the 3d FP32 displacement steps: node per thread (0) or
// component rows with 4 (1) or 3 (2) resident blocks of 384 threads per SM
// (at most 40 or 56 registers).  Chosen per operation (Chebyshev step or
// residual) and size class at the first call outside a stream capture by
// timing each variant on scratch vectors (the results are bit-identical, only
// the speed differs); PFF_STENCIL_VARIANT = 0 | 1 | 2 forces one.  The choice
// goes to the tuning record (PFF_TUNE_CACHE).
constexpr int N_VARIANTS = 3;
std::mutex g_variant_mu;
std::map<std::pair<int, int>, int> g_variant;   // (op: 0 Chebyshev, 1 residual, size class) -> variant

int forced_variant() {
  static const int f = [] {
    const char* e = std::getenv("PFF_STENCIL_VARIANT");
    if (!e) return -1;
    const int v = std::atoi(e);
    return v >= 0 && v < N_VARIANTS ? v : -1;
  }();
  return f;
}

template <bool RESID, int MINB>
void launch_rows3_b(const MeshDev& m, int64_t n, const float* K, const float* dinv, const float* rhs,
                    const float* xin, float* out, float* d, float cd, float cr, int zero_x,
                    const double* rhs64, float* rhs_store, double* out64, cudaStream_t s) {
  const unsigned g = grid_for(n, 32 * ROWS_GROUPS);
  if (stream_stencil(3, 3, 4, n))
    k_stencil_rows3<RESID, true, MINB><<<g, ROWS_THREADS, 0, s>>>(m, (int)n, K, dinv, rhs, xin, out, d,
                                                                cd, cr, zero_x, rhs64, rhs_store, out64);
  else
    k_stencil_rows3<RESID, false, MINB><<<g, ROWS_THREADS, 0, s>>>(m, (int)n, K, dinv, rhs, xin, out, d,
                                                                 cd, cr, zero_x, rhs64, rhs_store, out64);
}

// variant 1 or 2
template <bool RESID>
void launch_rows3(int variant, const MeshDev& m, int64_t n, const float* K, const float* dinv,
                  const float* rhs, const float* xin, float* out, float* d, float cd, float cr,
                  int zero_x, const double* rhs64, float* rhs_store, double* out64, cudaStream_t s) {
  if (variant == 1)
    launch_rows3_b<RESID, 4>(m, n, K, dinv, rhs, xin, out, d, cd, cr, zero_x, rhs64, rhs_store, out64, s);
  else
    launch_rows3_b<RESID, 3>(m, n, K, dinv, rhs, xin, out, d, cd, cr, zero_x, rhs64, rhs_store, out64, s);
}

int rows_variant(bool resid, const MeshDev& m, int64_t n, const float* K, cudaStream_t s) {
  const int f = forced_variant();
  if (f >= 0) return f;
  int cls = 0;
  while (cls < 62 && (int64_t(1) << (cls + 1)) <= n) ++cls;
  const auto key = std::make_pair(resid ? 1 : 0, cls);
  {
    std::lock_guard<std::mutex> g(g_variant_mu);
    auto it = g_variant.find(key);
    if (it != g_variant.end()) return it->second;
  }
  char rkey[64];
  std::snprintf(rkey, sizeof(rkey), "stencil_rows:%s:3:3:%d", resid ? "resid" : "cheb", cls);
  int recorded = 0;
  if (tune_lookup(rkey, &recorded) && recorded >= 0 && recorded < N_VARIANTS) {
    std::lock_guard<std::mutex> g(g_variant_mu);
    g_variant[key] = recorded;
    return recorded;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return 0;   // no timing inside a capture; decided at the next uncaptured call
  }
  // scratch x, rhs, output, inverse diagonal and Chebyshev direction (zeros)
  float* x = dalloc<float>(3 * n);
  float* b = dalloc<float>(3 * n);
  float* r = dalloc<float>(3 * n);
  float* dv = dalloc<float>(3 * n);
  float* dd = dalloc<float>(3 * n);
  for (float* v : {x, b, dv, dd}) PFF_CUDA(cudaMemsetAsync(v, 0, sizeof(float) * 3 * n, s));
  cudaEvent_t e0, e1;
  PFF_CUDA(cudaEventCreate(&e0));
  PFF_CUDA(cudaEventCreate(&e1));
  float ms[N_VARIANTS] = {0.f, 0.f, 0.f};
  for (int v = 0; v < N_VARIANTS; ++v) {
    auto run = [&]() {
      const unsigned g = grid_for(n, StencilShape<3, 3>::threads);
      constexpr int tb = StencilShape<3, 3>::threads;
      const bool sk = stream_stencil(3, 3, 4, n);
      if (resid) {
        if (v > 0)
          launch_rows3<true>(v, m, n, K, nullptr, b, x, r, nullptr, 0.f, 0.f, 0, nullptr, nullptr, nullptr, s);
        else if (sk)
          k_stencil_resid<float, 3, 3, true><<<g, tb, 0, s>>>(m, n, K, b, x, r);
        else
          k_stencil_resid<float, 3, 3, false><<<g, tb, 0, s>>>(m, n, K, b, x, r);
      } else {
        if (v > 0)
          launch_rows3<false>(v, m, n, K, dv, b, x, r, dd, 0.5f, 0.5f, 0, nullptr, nullptr, nullptr, s);
        else if (sk)
          k_stencil_cheb<float, 3, 3, true><<<g, tb, 0, s>>>(m, n, K, dv, b, x, r, dd, 0.5f, 0.5f, 0,
                                                              nullptr, nullptr, nullptr);
        else
          k_stencil_cheb<float, 3, 3, false><<<g, tb, 0, s>>>(m, n, K, dv, b, x, r, dd, 0.5f, 0.5f, 0,
                                                               nullptr, nullptr, nullptr);
      }
    };
    run();   // warm
    PFF_CUDA(cudaEventRecord(e0, s));
    run();
    run();
    PFF_CUDA(cudaEventRecord(e1, s));
    PFF_CUDA(cudaEventSynchronize(e1));
    PFF_LAUNCH("stencil variant tuning");
    PFF_CUDA(cudaEventElapsedTime(&ms[v], e0, e1));
  }
  count_launch(3 * N_VARIANTS);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (float* v : {x, b, r, dv, dd}) dfree(v);
  int best = 0;
  for (int v = 1; v < N_VARIANTS; ++v)
    if (ms[v] < ms[best]) best = v;
  if (verbose())
    std::fprintf(stderr, "[pff] stencil variant 3d %s n=%lld: node %.2f us, rows/4 %.2f us, rows/3 %.2f us -> %d\n",
                 resid ? "residual" : "Chebyshev", (long long)n, 500.0f * ms[0], 500.0f * ms[1],
                 500.0f * ms[2], best);
  tune_store(rkey, best);
  std::lock_guard<std::mutex> g(g_variant_mu);
  g_variant[key] = best;
  return best;
}
}  // namespace

#define STENCIL_LAUNCH_(D_, B_, SK, KERNEL, ...)                                        \
  KERNEL<T, D_, B_, SK><<<grid_for(n, StencilShape<D_, B_>::threads),                  \
                          StencilShape<D_, B_>::threads, 0, s>>>(__VA_ARGS__)
#define STENCIL_DISPATCH_SK(dim, b, SK, KERNEL, ...)                                    \
  do {                                                                                 \
    if ((dim) == 2 && (b) == 2) STENCIL_LAUNCH_(2, 2, SK, KERNEL, __VA_ARGS__);          \
    else if ((dim) == 2 && (b) == 1) STENCIL_LAUNCH_(2, 1, SK, KERNEL, __VA_ARGS__);     \
    else if ((dim) == 3 && (b) == 3) STENCIL_LAUNCH_(3, 3, SK, KERNEL, __VA_ARGS__);     \
    else if ((dim) == 3 && (b) == 1) STENCIL_LAUNCH_(3, 1, SK, KERNEL, __VA_ARGS__);     \
    else fail(PFF_ERR_INVALID_ARG, "stencil block size must be dim or 1");           \
  } while (0)
#define STENCIL_DISPATCH(dim, b, KERNEL, ...)                                         \
  do {                                                                                 \
    if (stream_stencil(dim, b, sizeof(T), n)) STENCIL_DISPATCH_SK(dim, b, true, KERNEL, __VA_ARGS__); \
    else STENCIL_DISPATCH_SK(dim, b, false, KERNEL, __VA_ARGS__);                      \
  } while (0)

template <class T>
void launch_stencil_cheb(const MeshDev& m, int64_t n, int b, const T* K, const T* dinv,
                         const T* rhs, const T* xin, T* xout, T* d, double cd, double cr,
                         int zero_x, cudaStream_t s, bool node_major, const double* rhs64,
                         T* rhs_store, double* out64) {
  if (rhs64 && !rhs_store) fail(PFF_ERR_INVALID_ARG, "stencil Chebyshev: FP64 rhs without a store");
  // stencil values (unless starting from zero), then dinv, rhs, x_in, x_out, d read + write;
  // an FP64 rhs adds its FP32 store and 4 bytes per read, an FP64 result replaces x_out and d
  const double bytes = sizeof(T) * (double)n *
                       ((zero_x ? 0.0 : slots_stored(m.dim, sizeof(T)) * b * b) + b * (zero_x ? 4.0 : 6.0)) +
                       (rhs64 ? 8.0 * n * b : 0.0) + (out64 ? (8.0 - 2.0 * sizeof(T)) * n * b : 0.0);
  // the displacement (b = dim) and phase-field (b = 1) smoothers are timed apart: their
  // V-cycles run concurrently on two streams
  ProfScope ps(sizeof(T) == 8 ? (b == 1 ? "cheb0_phi_f64" : "cheb0_u_f64")
                              : (b == 1 ? "cheb0_phi_f32" : "cheb0_u_f32"),
               bytes, s);
  if constexpr (sizeof(T) == 4) {
    if (node_major && m.dim == 2 && b == 2) {
      const unsigned g = grid_for(n, Q2_BLK);
      if (stream_stencil(2, 2, 4, n))
        k_stencil_cheb_q2<true><<<g, Q2_BLK, 0, s>>>(m, (int)n, K, dinv, rhs, xin, xout, d, (float)cd,
                                                     (float)cr, zero_x, rhs64, rhs_store, out64);
      else
        k_stencil_cheb_q2<false><<<g, Q2_BLK, 0, s>>>(m, (int)n, K, dinv, rhs, xin, xout, d, (float)cd,
                                                      (float)cr, zero_x, rhs64, rhs_store, out64);
      PFF_LAUNCH("stencil_cheb");
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    const int v = m.dim == 3 && b == 3 ? rows_variant(false, m, n, K, s) : 0;
    if (v > 0) {
      launch_rows3<false>(v, m, n, K, dinv, rhs, xin, xout, d, (float)cd, (float)cr, zero_x, rhs64,
                          rhs_store, out64, s);
      PFF_LAUNCH("stencil_cheb");
      return;
    }
  }
  STENCIL_DISPATCH(m.dim, b, k_stencil_cheb, m, n, K, dinv, rhs, xin, xout, d, (T)cd, (T)cr, zero_x,
                   rhs64, rhs_store, out64);
  PFF_LAUNCH("stencil_cheb");
}

template <class T>
void launch_stencil_resid(const MeshDev& m, int64_t n, int b, const T* K, const T* rhs, const T* x,
                          T* r, cudaStream_t s, bool node_major) {
  const double bytes = sizeof(T) * (double)n * (slots_stored(m.dim, sizeof(T)) * b * b + 3.0 * b);
  ProfScope ps(sizeof(T) == 8 ? (b == 1 ? "resid0_phi_f64" : "resid0_u_f64")
                              : (b == 1 ? "resid0_phi_f32" : "resid0_u_f32"),
               bytes, s);
  if constexpr (sizeof(T) == 4) {
    if (node_major && m.dim == 2 && b == 2) {
      const unsigned g = grid_for(n, Q2_BLK);
      if (stream_stencil(2, 2, 4, n))
        k_stencil_resid_q2<true><<<g, Q2_BLK, 0, s>>>(m, (int)n, K, rhs, x, r);
      else
        k_stencil_resid_q2<false><<<g, Q2_BLK, 0, s>>>(m, (int)n, K, rhs, x, r);
      PFF_LAUNCH("stencil_resid");
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    const int v = m.dim == 3 && b == 3 ? rows_variant(true, m, n, K, s) : 0;
    if (v > 0) {
      launch_rows3<true>(v, m, n, K, nullptr, rhs, x, r, nullptr, 0.f, 0.f, 0, nullptr, nullptr, nullptr, s);
      PFF_LAUNCH("stencil_resid");
      return;
    }
  }
  STENCIL_DISPATCH(m.dim, b, k_stencil_resid, m, n, K, rhs, x, r);
  PFF_LAUNCH("stencil_resid");
}

template void launch_stencil_cheb<float>(const MeshDev&, int64_t, int, const float*, const float*,
                                         const float*, const float*, float*, float*, double, double,
                                         int, cudaStream_t, bool, const double*, float*, double*);
template void launch_stencil_cheb<double>(const MeshDev&, int64_t, int, const double*,
                                          const double*, const double*, const double*, double*,
                                          double*, double, double, int, cudaStream_t, bool,
                                          const double*, double*, double*);
template void launch_stencil_resid<float>(const MeshDev&, int64_t, int, const float*, const float*,
                                          const float*, float*, cudaStream_t, bool);
template void launch_stencil_resid<double>(const MeshDev&, int64_t, int, const double*,
                                           const double*, const double*, double*, cudaStream_t, bool);

void stencil_to_node_major(const double* K, float* Kq, int64_t n, cudaStream_t s) {
  ProfScope ps("to_f32", 48.0 * 5 * n, s);
  k_stencil_to_q2<<<grid_for(5 * n, 256), 256, 0, s>>>(n, K, Kq);
  PFF_LAUNCH("stencil_to_q2");
}

int64_t stencil_f32_count(int dim, int b, int64_t n) {
  const int64_t nh = dim == 2 ? 5 : 14;
  return nh * b * b * n;
}

void stencil_to_f32(int dim, int b, const double* K, float* Kf, int64_t n, cudaStream_t s) {
  // slot-major: the stored slots C..3^d-1 are one contiguous range of K
  const int64_t c = dim == 2 ? 4 : 13;
  convert_d2f(K + c * b * b * n, Kf, stencil_f32_count(dim, b, n), s);
}

void launch_stencil_dinv(const MeshDev& m, int64_t n, int b, const double* K, double* dinv,
                         float* dinvf, cudaStream_t s) {
  ProfScope ps("stencil_dinv", (double)n * b * (8.0 + 8.0 + (dinvf ? 4.0 : 0.0)), s);
  k_stencil_dinv<<<grid_for(n, 256), 256, 0, s>>>(n, b, m.dim == 2 ? 4 : 13, K, dinv, dinvf);
  PFF_LAUNCH("stencil_dinv");
}

}  // namespace pff
