// Vector-BSR kernels of the AMG hierarchy (Section 3.1: each preconditioner
// block is one smoothed-aggregation V-cycle; its coarse operators, prolongators
// and restrictions are block-sparse).
//
// A group of G lanes (G | 32) works on one block row.  Per pass the group
// takes G consecutive blocks of the row: for G >= 4 their values, which are
// contiguous in memory, are read by the whole group with unit stride into
// shared memory, and lane j then multiplies block j with its gathered x block
// (G = 1, 2 suit rows of one or two blocks: each lane reads its own blocks).
// The G partial row sums are combined with xor shuffles inside the group, and
// lanes 0..BR-1 run the epilogue of the block row's BR scalar rows:
//   OP_SPMV   y = alpha A x + beta y
//   OP_RESID  y = rhs - A x
//   OP_CHEB   one Chebyshev step: d = cd d + cr D^-1 (rhs - A x); xout = x + d
// The SELL-32 kernels keep one thread per block row: the blocks of 32
// consecutive rows are stored entry-major (block k of the 32 rows, then block
// k + 1, ...), so every value and column load of a warp reads 128 contiguous
// bytes, and no shuffles or staging are needed; a row shorter than its slice's
// longest row simply stops early (the padding is never read).
// The row-per-thread kernels on the plain BSR arrays (one scalar row per
// thread, uncoalesced value reads) stay available as the reference variant
// (Bsr::group = -1).
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "pff_internal.h"

namespace pff {
namespace {

enum { OP_SPMV = 0, OP_RESID = 1, OP_CHEB = 2 };

template <class T>
struct VecArgs {
  int nrows;
  const int* __restrict__ rp;
  const int* __restrict__ col;
  const T* __restrict__ val;
  const T* __restrict__ x;
  T* y;                          // SPMV / RESID output; CHEB: xout
  const T* __restrict__ rhs;
  const T* __restrict__ dinv;
  T* d;
  T alpha, beta;                 // SPMV scalars; CHEB: cd, cr
};

__host__ __device__ constexpr int threads_for(int bb) { return bb >= 16 ? 128 : 256; }

template <class T, int BR, int BC, int G, int OP>
__global__ void __launch_bounds__(threads_for(BR * BC))
    k_bsr_vec(VecArgs<T> p) {
  constexpr int BB = BR * BC;
  constexpr int NT = threads_for(BB);
  constexpr int NG = NT / G;
  constexpr bool STAGE = BB > 1 && G >= 4;
  __shared__ T sv[STAGE ? NT * BB : 1];
  const int grp = threadIdx.x / G, lane = threadIdx.x % G;
  const unsigned gmask = G == 32 ? 0xffffffffu
                                 : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const int I = blockIdx.x * NG + grp;
  const bool valid = I < p.nrows;
  T s[BR];
#pragma unroll
  for (int a = 0; a < BR; ++a) s[a] = T(0);
  int k0 = 0, k1 = 0;
  if (valid) {
    k0 = p.rp[I];
    k1 = p.rp[I + 1];
  }
  T* my = sv + (STAGE ? grp * G * BB : 0);
  for (int kb = k0; kb < k1; kb += G) {   // trip count is uniform within a group
    const int nb = min(G, k1 - kb);
    if constexpr (STAGE) {
      const T* src = p.val + (int64_t)kb * BB;
      for (int e = lane; e < nb * BB; e += G) my[e] = src[e];
      __syncwarp(gmask);
    }
    if (lane < nb) {
      const int c = p.col[kb + lane];
      const T* xx = p.x + (int64_t)c * BC;
      T xv[BC];
#pragma unroll
      for (int cc = 0; cc < BC; ++cc) xv[cc] = xx[cc];
      const T* v = STAGE ? my + lane * BB : p.val + (int64_t)(kb + lane) * BB;
#pragma unroll
      for (int a = 0; a < BR; ++a)
#pragma unroll
        for (int cc = 0; cc < BC; ++cc) s[a] += v[a * BC + cc] * xv[cc];
    }
    if constexpr (STAGE) __syncwarp(gmask);
  }
  // every lane of the warp reaches the shuffles (no early return above)
#pragma unroll
  for (int a = 0; a < BR; ++a)
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s[a] += __shfl_xor_sync(0xffffffffu, s[a], o);
  if (!valid) return;
#pragma unroll
  for (int a = 0; a < BR; ++a) {
    if (a % G != lane) continue;
    const int64_t r = (int64_t)I * BR + a;
    if constexpr (OP == OP_SPMV) {
      p.y[r] = p.beta == T(0) ? p.alpha * s[a] : p.alpha * s[a] + p.beta * p.y[r];
    } else if constexpr (OP == OP_RESID) {
      p.y[r] = p.rhs[r] - s[a];
    } else {
      const T res = p.dinv[r] * (p.rhs[r] - s[a]);
      const T dn = p.alpha * p.d[r] + p.beta * res;
      p.d[r] = dn;
      p.y[r] = p.x[r] + dn;
    }
  }
}

template <class T, int BR, int BC, int OP>
bool launch_g(int G, const VecArgs<T>& a, cudaStream_t s) {
  constexpr int NT = threads_for(BR * BC);
  const unsigned grid = (unsigned)((a.nrows + NT / G - 1) / (NT / G));
  switch (G) {
    case 1: k_bsr_vec<T, BR, BC, 1, OP><<<grid, NT, 0, s>>>(a); return true;
    case 2: k_bsr_vec<T, BR, BC, 2, OP><<<grid, NT, 0, s>>>(a); return true;
    case 4: k_bsr_vec<T, BR, BC, 4, OP><<<grid, NT, 0, s>>>(a); return true;
    case 8: k_bsr_vec<T, BR, BC, 8, OP><<<grid, NT, 0, s>>>(a); return true;
    case 16: k_bsr_vec<T, BR, BC, 16, OP><<<grid, NT, 0, s>>>(a); return true;
    case 32: k_bsr_vec<T, BR, BC, 32, OP><<<grid, NT, 0, s>>>(a); return true;
    default: return false;
  }
}

template <class T, int OP>
bool launch_shape(int br, int bc, int G, const VecArgs<T>& a, cudaStream_t s) {
  const int key = br * 10 + bc;
  if constexpr (OP == OP_SPMV) {
    switch (key) {
      case 23: return launch_g<T, 2, 3, OP>(G, a, s);
      case 32: return launch_g<T, 3, 2, OP>(G, a, s);
      case 36: return launch_g<T, 3, 6, OP>(G, a, s);
      case 63: return launch_g<T, 6, 3, OP>(G, a, s);
      default: break;
    }
  }
  switch (key) {
    case 11: return launch_g<T, 1, 1, OP>(G, a, s);
    case 22: return launch_g<T, 2, 2, OP>(G, a, s);
    case 33: return launch_g<T, 3, 3, OP>(G, a, s);
    case 66: return launch_g<T, 6, 6, OP>(G, a, s);
    default: return false;
  }
}

// ------------------------------------------------------------ SELL-32 ---
struct SellArgs {
  int nrows;
  const int* __restrict__ rp;     // BSR row pointers: the row lengths
  const int* __restrict__ off;    // slice offsets (entry columns)
  const int* __restrict__ scol;
  const float* __restrict__ sval;
  const float* __restrict__ x;
  float* y;
  const float* __restrict__ rhs;
  const float* __restrict__ dinv;
  float* d;
  float alpha, beta;
};

template <int BR, int BC, int OP>
__global__ void __launch_bounds__(256) k_sell(SellArgs p) {
  constexpr int BB = BR * BC;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= p.nrows) return;
  const int l = row & 31;
  const int64_t base = p.off[row >> 5];
  const int len = p.rp[row + 1] - p.rp[row];
  const int* cp = p.scol + base * 32 + l;
  const float* vp = p.sval + base * BB * 32 + l;
  float s[BR];
#pragma unroll
  for (int a = 0; a < BR; ++a) s[a] = 0.f;
#pragma unroll 2
  for (int k = 0; k < len; ++k) {
    const int c = cp[k * 32];
    float xv[BC];
#pragma unroll
    for (int cc = 0; cc < BC; ++cc) xv[cc] = p.x[(int64_t)c * BC + cc];
#pragma unroll
    for (int a = 0; a < BR; ++a)
#pragma unroll
      for (int cc = 0; cc < BC; ++cc) s[a] += vp[(k * BB + a * BC + cc) * 32] * xv[cc];
  }
#pragma unroll
  for (int a = 0; a < BR; ++a) {
    const int64_t r = (int64_t)row * BR + a;
    if constexpr (OP == OP_SPMV) {
      p.y[r] = p.beta == 0.f ? p.alpha * s[a] : p.alpha * s[a] + p.beta * p.y[r];
    } else if constexpr (OP == OP_RESID) {
      p.y[r] = p.rhs[r] - s[a];
    } else {
      const float res = p.dinv[r] * (p.rhs[r] - s[a]);
      const float dn = p.alpha * p.d[r] + p.beta * res;
      p.d[r] = dn;
      p.y[r] = p.x[r] + dn;
    }
  }
}

template <int OP>
bool launch_sell(int br, int bc, const SellArgs& a, cudaStream_t s) {
  const unsigned grid = (unsigned)((a.nrows + 255) / 256);
  const int key = br * 10 + bc;
  if constexpr (OP == OP_SPMV) {
    switch (key) {
      case 23: k_sell<2, 3, OP><<<grid, 256, 0, s>>>(a); return true;
      case 32: k_sell<3, 2, OP><<<grid, 256, 0, s>>>(a); return true;
      case 36: k_sell<3, 6, OP><<<grid, 256, 0, s>>>(a); return true;
      case 63: k_sell<6, 3, OP><<<grid, 256, 0, s>>>(a); return true;
      default: break;
    }
  }
  switch (key) {
    case 11: k_sell<1, 1, OP><<<grid, 256, 0, s>>>(a); return true;
    case 22: k_sell<2, 2, OP><<<grid, 256, 0, s>>>(a); return true;
    case 33: k_sell<3, 3, OP><<<grid, 256, 0, s>>>(a); return true;
    case 66: k_sell<6, 6, OP><<<grid, 256, 0, s>>>(a); return true;
    default: return false;
  }
}

// longest row of each slice of 32 block rows
__global__ void k_sell_len(int nrows, const int* __restrict__ rp, int* __restrict__ len) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = row < nrows ? rp[row + 1] - rp[row] : 0;
  const int m = __reduce_max_sync(0xffffffffu, l);
  if ((threadIdx.x & 31) == 0 && row < nrows) len[row >> 5] = m;
}

__global__ void k_sell_fill(int nrows, int bb, const int* __restrict__ rp,
                            const int* __restrict__ col, const double* __restrict__ val,
                            const int* __restrict__ off, int* __restrict__ scol,
                            float* __restrict__ sval) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrows) return;
  const int l = row & 31;
  const int64_t base = off[row >> 5];
  const int k0 = rp[row], len = rp[row + 1] - k0;
  for (int k = 0; k < len; ++k) {
    scol[(base + k) * 32 + l] = col[k0 + k];
    for (int e = 0; e < bb; ++e)
      sval[((base + k) * bb + e) * 32 + l] = (float)val[(int64_t)(k0 + k) * bb + e];
  }
}

// ------------------------------------------- row-per-thread reference ---
template <class T>
__global__ void k_row_spmv(int nrows, int br, int bc, const int* __restrict__ rowptr,
                           const int* __restrict__ col, const T* __restrict__ val,
                           const T* __restrict__ x, T* __restrict__ y, T alpha, T beta) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (int64_t)nrows * br) return;
  const int I = (int)(r / br), a = (int)(r % br);
  T s = 0;
  for (int k = rowptr[I]; k < rowptr[I + 1]; ++k) {
    const T* v = val + ((int64_t)k * br + a) * bc;
    const T* xx = x + (int64_t)col[k] * bc;
    for (int c = 0; c < bc; ++c) s += v[c] * xx[c];
  }
  y[r] = beta == T(0) ? alpha * s : alpha * s + beta * y[r];
}

template <class T>
__global__ void k_row_resid(int n, int b, const int* __restrict__ rp, const int* __restrict__ col,
                            const T* __restrict__ val, const T* __restrict__ rhs,
                            const T* __restrict__ x, T* __restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * b) return;
  const int I = (int)(i / b), a = (int)(i % b);
  T s = 0;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const T* v = val + ((int64_t)k * b + a) * b;
    const T* xx = x + (int64_t)col[k] * b;
    for (int c = 0; c < b; ++c) s += v[c] * xx[c];
  }
  r[i] = rhs[i] - s;
}

// zero_x: the first step from x = 0 needs no product
template <class T>
__global__ void k_row_cheb(int n, int b, const int* __restrict__ rp, const int* __restrict__ col,
                           const T* __restrict__ val, const T* __restrict__ dinv,
                           const T* __restrict__ rhs, const T* __restrict__ xin, T* __restrict__ xout,
                           T* __restrict__ d, T cd, T cr, int zero_x) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (int64_t)n * b) return;
  T s = 0;
  if (!zero_x) {
    const int I = (int)(r / b), a = (int)(r % b);
    for (int k = rp[I]; k < rp[I + 1]; ++k) {
      const T* v = val + ((int64_t)k * b + a) * b;
      const T* xx = xin + (int64_t)col[k] * b;
      for (int c = 0; c < b; ++c) s += v[c] * xx[c];
    }
  }
  const T res = dinv[r] * (rhs[r] - s);
  const T dn = cd * (zero_x ? T(0) : d[r]) + cr * res;
  d[r] = dn;
  xout[r] = (zero_x ? T(0) : xin[r]) + dn;
}

template <class T>
const T* values(const Bsr& A) {
  if constexpr (sizeof(T) == 8) return reinterpret_cast<const T*>(A.val);
  else return reinterpret_cast<const T*>(A.valf);
}

}  // namespace

void bsr_make_sell(Bsr& A, cudaStream_t s) {
  dfree(A.sell_off);
  dfree(A.sell_col);
  dfree(A.sell_valf);
  A.sell_off = A.sell_col = nullptr;
  A.sell_valf = nullptr;
  if (A.nrows == 0) return;
  const int ns = (A.nrows + 31) / 32;
  int* len = dalloc<int>(ns + 1);
  A.sell_off = dalloc<int>(ns + 1);
  count_launch();
  k_sell_len<<<(ns * 32 + 255) / 256, 256, 0, s>>>(A.nrows, A.rowptr, len);
  int cols = 0;
  exclusive_scan_int(len, A.sell_off, ns, &cols, s);
  const int64_t entries = (int64_t)cols * 32;
  const int bb = A.br * A.bc;
  A.sell_col = dalloc<int>(std::max<int64_t>(entries, 1));
  A.sell_valf = dalloc<float>(std::max<int64_t>(entries * bb, 1));
  count_launch();
  k_sell_fill<<<grid_for(A.nrows, 256), 256, 0, s>>>(A.nrows, bb, A.rowptr, A.col, A.val,
                                                     A.sell_off, A.sell_col, A.sell_valf);
  PFF_LAUNCH("sell");
  PFF_CUDA(cudaStreamSynchronize(s));
  dfree(len);
}

namespace {
// launch OP through the SELL copy (FP32 only); false when it cannot be used
template <class T, int OP>
bool sell_op(const Bsr& A, const T* x, T* y, const T* rhs, const T* dinv, T* d, T alpha, T beta,
             cudaStream_t s) {
  if constexpr (sizeof(T) != 4) {
    return false;
  } else {
    if (!A.sell_valf) return false;
    SellArgs a{A.nrows, A.rowptr, A.sell_off, A.sell_col, A.sell_valf, x, y, rhs, dinv, d,
               alpha, beta};
    return launch_sell<OP>(A.br, A.bc, a, s);
  }
}
}  // namespace

// ------------------------------------------------------------ autotune ---
// The lane-group width of each hierarchy matrix is picked by timing every
// candidate on that matrix once; the winner is remembered per (element size,
// block shape, log2 rows, half-log2 mean row length), so the hierarchies
// rebuilt at later loading steps reuse it without timing.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune;

template <class T>
int tune_one(Bsr& A, cudaStream_t s) {
  const double avg = A.nrows > 0 ? (double)A.nnzb / A.nrows : 1.0;
  const auto key = std::make_tuple((int)sizeof(T), A.br * 10 + A.bc,
                                   (int)std::floor(std::log2(std::max(1, A.nrows))),
                                   (int)std::lround(2.0 * std::log2(std::max(1.0, avg))), 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      if (it->second == BSR_SELL) bsr_make_sell(A, s);
      return it->second;
    }
  }
  char rkey[96];
  std::snprintf(rkey, sizeof(rkey), "spmv:%d:%d:%d:%d", std::get<0>(key), std::get<1>(key),
                std::get<2>(key), std::get<3>(key));
  int recorded = 0;
  if (tune_lookup(rkey, &recorded)) {
    if (recorded == BSR_SELL) bsr_make_sell(A, s);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = recorded;
    return recorded;
  }
  const int64_t nx = (int64_t)A.ncols * A.bc, ny = (int64_t)A.nrows * A.br;
  T* x = dalloc<T>(nx);
  T* y = dalloc<T>(ny);
  PFF_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * nx, s));
  cudaEvent_t e0, e1;
  PFF_CUDA(cudaEventCreate(&e0));
  PFF_CUDA(cudaEventCreate(&e1));
  VecArgs<T> a{A.nrows, A.rowptr, A.col, values<T>(A), x, y, nullptr, nullptr, nullptr, T(1), T(0)};
  int best = 4;
  float best_ms = 1e30f;
  if constexpr (sizeof(T) == 4) bsr_make_sell(A, s);
  for (int G : {1, 2, 4, 8, 16, 32, (int)BSR_SELL}) {
    auto run = [&]() {
      return G == BSR_SELL ? sell_op<T, OP_SPMV>(A, x, y, (const T*)nullptr, (const T*)nullptr,
                                                 (T*)nullptr, T(1), T(0), s)
                           : launch_shape<T, OP_SPMV>(A.br, A.bc, G, a, s);
    };
    count_launch(4);
    if (!run()) continue;   // shape or precision without this variant
    PFF_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 3; ++r) run();
    PFF_CUDA(cudaEventRecord(e1, s));
    PFF_CUDA(cudaEventSynchronize(e1));
    PFF_LAUNCH("spmv autotune");
    float ms = 0.f;
    PFF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (verbose())
      std::fprintf(stderr, "[pff] spmv tune %dx%d rows %d nnzb %lld variant %d: %.2f us %.0f GB/s\n",
                   A.br, A.bc, A.nrows, (long long)A.nnzb, G, 1e3 * ms / 3,
                   bsr_bytes(A, sizeof(T), false) / (ms / 3 * 1e-3) * 1e-9);
    if (ms < best_ms) {
      best_ms = ms;
      best = G;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PFF_CUDA(cudaStreamSynchronize(s));
  dfree(x);
  dfree(y);
  if (best != BSR_SELL) {   // keep the sliced copy only where it is used
    dfree(A.sell_off);
    dfree(A.sell_col);
    dfree(A.sell_valf);
    A.sell_off = A.sell_col = nullptr;
    A.sell_valf = nullptr;
  }
  tune_store(rkey, best);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}
}  // namespace

void bsr_autotune(Bsr& A, bool f32, cudaStream_t s) {
  if (A.nrows == 0 || A.nnzb == 0) return;
  A.group = f32 ? tune_one<float>(A, s) : tune_one<double>(A, s);
}

namespace {
// one pass over an average row: the smallest power of two >= mean blocks per row
int group_by_length(const Bsr& A) {
  const double avg = A.nrows > 0 ? (double)A.nnzb / A.nrows : 1.0;
  int g = 4;
  while (g < 32 && g < avg) g *= 2;
  return g;
}
}  // namespace

int bsr_group(const Bsr& A) { return A.group != 0 ? A.group : group_by_length(A); }

double bsr_bytes(const Bsr& A, int elem, bool beta) {
  return (double)A.nnzb * (A.br * A.bc * (double)elem + 4.0) + 4.0 * (A.nrows + 1.0) +
         (double)elem * ((double)A.ncols * A.bc + (double)A.nrows * A.br * (beta ? 2.0 : 1.0));
}

template <class T>
void bsr_spmv_t(const Bsr& A, const T* x, T* y, T alpha, T beta, cudaStream_t s) {
  const int64_t rows = (int64_t)A.nrows * A.br;
  if (rows == 0) return;
  ProfScope ps(sizeof(T) == 8 ? "spmv_f64" : "spmv_f32", bsr_bytes(A, sizeof(T), beta != T(0)), s);
  int G = bsr_group(A);
  if (G == BSR_SELL && sell_op<T, OP_SPMV>(A, x, y, (const T*)nullptr, (const T*)nullptr,
                                           (T*)nullptr, alpha, beta, s)) {
    PFF_LAUNCH("bsr_spmv");
    return;
  }
  if (G == BSR_SELL) G = group_by_length(A);
  VecArgs<T> a{A.nrows, A.rowptr, A.col, values<T>(A), x, y, nullptr, nullptr, nullptr, alpha, beta};
  if (G < 0 || !launch_shape<T, OP_SPMV>(A.br, A.bc, G, a, s))
    k_row_spmv<T><<<grid_for(rows, 256), 256, 0, s>>>(A.nrows, A.br, A.bc, A.rowptr, A.col,
                                                       values<T>(A), x, y, alpha, beta);
  PFF_LAUNCH("bsr_spmv");
}

void bsr_spmv(const Bsr& A, const double* x, double* y, double alpha, double beta, cudaStream_t s) {
  bsr_spmv_t<double>(A, x, y, alpha, beta, s);
}

void bsr_spmv_f(const Bsr& A, const float* x, float* y, float alpha, float beta, cudaStream_t s) {
  bsr_spmv_t<float>(A, x, y, alpha, beta, s);
}

template <class T>
void bsr_resid(const Bsr& A, const T* rhs, const T* x, T* r, cudaStream_t s) {
  const int64_t rows = (int64_t)A.nrows * A.br;
  if (rows == 0) return;
  ProfScope ps(sizeof(T) == 8 ? "resid_f64" : "resid_f32",
               (double)A.nnzb * (A.br * A.bc * (double)sizeof(T) + 4.0) + 4.0 * (A.nrows + 1.0) +
                   3.0 * sizeof(T) * (double)rows, s);
  int G = bsr_group(A);
  if (G == BSR_SELL && A.br == A.bc &&
      sell_op<T, OP_RESID>(A, x, r, rhs, (const T*)nullptr, (T*)nullptr, T(0), T(0), s)) {
    PFF_LAUNCH("bsr_resid");
    return;
  }
  if (G == BSR_SELL) G = group_by_length(A);
  VecArgs<T> a{A.nrows, A.rowptr, A.col, values<T>(A), x, r, rhs, nullptr, nullptr, T(0), T(0)};
  if (G < 0 || A.br != A.bc || !launch_shape<T, OP_RESID>(A.br, A.bc, G, a, s))
    k_row_resid<T><<<grid_for(rows, 256), 256, 0, s>>>(A.nrows, A.br, A.rowptr, A.col,
                                                        values<T>(A), rhs, x, r);
  PFF_LAUNCH("bsr_resid");
}

template <class T>
void bsr_cheb(const Bsr& A, const T* dinv, const T* rhs, const T* xin, T* xout, T* d, T cd, T cr,
              bool zero_x, cudaStream_t s) {
  const int64_t rows = (int64_t)A.nrows * A.br;
  if (rows == 0) return;
  const double mat_b = (double)A.nnzb * (A.br * A.bc * (double)sizeof(T) + 4.0) + 4.0 * (A.nrows + 1.0);
  const double nvec = (double)rows * sizeof(T);
  ProfScope ps(sizeof(T) == 8 ? "cheb_f64" : "cheb_f32",
               (zero_x ? 0.0 : mat_b) + nvec * (zero_x ? 4.0 : 6.0), s);
  int G = bsr_group(A);
  if (!zero_x && G == BSR_SELL && A.br == A.bc &&
      sell_op<T, OP_CHEB>(A, xin, xout, rhs, dinv, d, cd, cr, s)) {
    PFF_LAUNCH("bsr_cheb");
    return;
  }
  if (G == BSR_SELL) G = group_by_length(A);
  VecArgs<T> a{A.nrows, A.rowptr, A.col, values<T>(A), xin, xout, rhs, dinv, d, cd, cr};
  if (zero_x || G < 0 || A.br != A.bc || !launch_shape<T, OP_CHEB>(A.br, A.bc, G, a, s))
    k_row_cheb<T><<<grid_for(rows, 256), 256, 0, s>>>(A.nrows, A.br, A.rowptr, A.col, values<T>(A),
                                                       dinv, rhs, xin, xout, d, cd, cr,
                                                       zero_x ? 1 : 0);
  PFF_LAUNCH("bsr_cheb");
}

template void bsr_resid<float>(const Bsr&, const float*, const float*, float*, cudaStream_t);
template void bsr_resid<double>(const Bsr&, const double*, const double*, double*, cudaStream_t);
template void bsr_cheb<float>(const Bsr&, const float*, const float*, const float*, float*, float*,
                              float, float, bool, cudaStream_t);
template void bsr_cheb<double>(const Bsr&, const double*, const double*, const double*, double*,
                               double*, double, double, bool, cudaStream_t);

}  // namespace pff
