// Smoothed-aggregation algebraic multigrid, built and applied on the device.
//
// Section 3.1 preconditions each diagonal block (M_uu: linear elasticity;
// M_phi_phi: mass + Laplacian) with one AMG V-cycle.  The paper uses Trilinos
// ML; this is an independent GPU design:
//   setup (per level, all on the device, deterministic):
//     1. strength graph: block (I,J) is strong iff ||A_IJ||_F^2 > theta^2
//        ||A_II||_F ||A_JJ||_F, symmetrized; rows without strong off-diagonal
//        blocks (Dirichlet / active identity rows, kappa-degenerate crack
//        nodes) are isolated and left to the smoother
//     2. aggregation: distance-2 maximal independent set (hash-keyed parallel
//        MIS(2)) as roots; every node joins the root it is most strongly
//        connected to, or else the aggregate of its most strongly connected
//        neighbour
//     3. tentative prolongator: per-aggregate thin QR (modified Gram-Schmidt,
//        twice) of the near-null space (rigid-body modes / constants); R gives
//        the coarse near-null space
//     4. P = (I - omega D_F^-1 A_F) P_tent, omega = 4 / (3 lambda_max(D^-1 A)),
//        A_F = A with weak off-diagonal blocks lumped into the diagonal block
//     5. R = P^T, A_c = R A P (two row-wise SpGEMMs with sorted unique columns)
//     6. coarsest level: dense inverse (Gauss-Jordan with partial pivoting)
//   V-cycle: Chebyshev(D^-1 A) pre/post smoothing, restriction, coarse solve,
//   prolongation; FP64 or FP32 (mixed precision) values and vectors.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <memory>

#include "pff_internal.h"

namespace pff {

namespace {

constexpr int CAP = 512;   // per-row unique-column capacity of the setup SpGEMMs

enum : int { ST_OUT = 0, ST_UND = 1, ST_IN = 2 };

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__device__ __forceinline__ unsigned long long mis_key(int state, int i) {
  return ((unsigned long long)state << 62) |
         ((unsigned long long)(hash32((uint32_t)i) & 0x3fffffffU) << 32) | (unsigned)i;
}

// -------------------------------------------------------------- diagonals --
__global__ void k_diag(int n, int b, const int* __restrict__ rp, const int* __restrict__ col,
                       const double* __restrict__ val, double* __restrict__ dnorm,
                       double* __restrict__ dinv, int* __restrict__ err) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int kd = -1;
  for (int k = rp[I]; k < rp[I + 1]; ++k)
    if (col[k] == I) {
      kd = k;
      break;
    }
  if (kd < 0) {
    atomicExch(err, 1);
    dnorm[I] = 0.0;
    for (int a = 0; a < b; ++a) dinv[(int64_t)I * b + a] = 0.0;
    return;
  }
  const double* v = val + (int64_t)kd * b * b;
  double s = 0.0;
  for (int e = 0; e < b * b; ++e) s += v[e] * v[e];
  dnorm[I] = sqrt(s);
  for (int a = 0; a < b; ++a) {
    const double dv = v[a * b + a];
    dinv[(int64_t)I * b + a] = dv != 0.0 ? 1.0 / dv : 0.0;
  }
}

// ---------------------------------------------------------------- strength --
__global__ void k_strength(int n, int b, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ dnorm,
                           double theta2, uint8_t* __restrict__ strong, double* __restrict__ snorm) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    const double* v = val + (int64_t)k * b * b;
    double s = 0.0;
    for (int e = 0; e < b * b; ++e) s += v[e] * v[e];
    snorm[k] = s;
    strong[k] = (J != I) && (s > theta2 * dnorm[I] * dnorm[J]);
  }
}

// Distance-Laplacian strength (for meshes with stretched cells, where the Q1
// matrix entries of the weak direction stay O(aspect ratio)): w_IJ = 1/|x_I -
// x_J|^2, strong iff w_IJ^2 >= theta^2 wmax_I wmax_J, and the matrix block is
// not negligible, ||A_IJ||^2 > mdrop^2 ||A_II|| ||A_JJ|| (this keeps the
// couplings of kappa-degenerate crack nodes and eliminated columns weak).
__device__ __forceinline__ double dist_w(const double* __restrict__ X, int cd, int I, int J) {
  double d2 = 0.0;
  for (int l = 0; l < cd; ++l) {
    const double t = X[(int64_t)I * cd + l] - X[(int64_t)J * cd + l];
    d2 += t * t;
  }
  return d2 > 0.0 ? 1.0 / d2 : 1e300;
}

__global__ void k_dist_wmax(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ X, int cd, double* __restrict__ wmax) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  double m = 0.0;
  for (int k = rp[I]; k < rp[I + 1]; ++k)
    if (col[k] != I) m = fmax(m, dist_w(X, cd, I, col[k]));
  wmax[I] = m;
}

__global__ void k_strength_dist(int n, int b, const int* __restrict__ rp, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ dnorm,
                                const double* __restrict__ X, int cd,
                                const double* __restrict__ wmax, double theta2, double mdrop2,
                                uint8_t* __restrict__ strong, double* __restrict__ snorm) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    if (J == I) {
      strong[k] = 0;
      snorm[k] = 0.0;
      continue;
    }
    const double* v = val + (int64_t)k * b * b;
    double m = 0.0;
    for (int e = 0; e < b * b; ++e) m += v[e] * v[e];
    const double w = dist_w(X, cd, I, J);
    const bool s = (w * w >= theta2 * wmax[I] * wmax[J]) && (m > mdrop2 * dnorm[I] * dnorm[J]);
    strong[k] = s;
    snorm[k] = w;
  }
}

// coarse-level coordinates: centroid of each aggregate's members
__global__ void k_centroids(int nagg, const int* __restrict__ off, const int* __restrict__ members,
                            const double* __restrict__ X, int cd, double* __restrict__ Xc) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nagg) return;
  const int lo = off[a], hi = off[a + 1];
  for (int l = 0; l < cd; ++l) {
    double s = 0.0;
    for (int t = lo; t < hi; ++t) s += X[(int64_t)members[t] * cd + l];
    Xc[(int64_t)a * cd + l] = hi > lo ? s / (hi - lo) : 0.0;
  }
}

__device__ __forceinline__ int find_col(const int* __restrict__ col, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int v = col[mid];
    if (v == c) return mid;
    if (v < c) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

// union with the transpose: out[k] = in[k] | in[k^T]
__global__ void k_symmetrize(int n, const int* __restrict__ rp, const int* __restrict__ col,
                             const uint8_t* __restrict__ in, uint8_t* __restrict__ out) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    uint8_t s = in[k];
    if (!s && J != I) {
      const int kt = find_col(col, rp[J], rp[J + 1], I);
      if (kt >= 0) s = in[kt];
    }
    out[k] = s;
  }
}

// -------------------------------------------------------------------- MIS --
__global__ void k_mis_init(int n, const int* __restrict__ rp, const uint8_t* __restrict__ strong,
                           int* __restrict__ state, uint8_t* __restrict__ iso) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  bool any = false;
  for (int k = rp[I]; k < rp[I + 1]; ++k) any |= strong[k] != 0;
  iso[I] = !any;
  state[I] = any ? ST_UND : ST_OUT;
}

__global__ void k_mis_max1(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const uint8_t* __restrict__ strong, const int* __restrict__ state,
                           unsigned long long* __restrict__ M1) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  unsigned long long m = mis_key(state[I], I);
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    if (!strong[k]) continue;
    const int J = col[k];
    const unsigned long long kj = mis_key(state[J], J);
    m = kj > m ? kj : m;
  }
  M1[I] = m;
}

__global__ void k_mis_max2(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const uint8_t* __restrict__ strong,
                           const unsigned long long* __restrict__ M1,
                           unsigned long long* __restrict__ M2) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  unsigned long long m = M1[I];
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    if (!strong[k]) continue;
    const unsigned long long kj = M1[col[k]];
    m = kj > m ? kj : m;
  }
  M2[I] = m;
}

__global__ void k_mis_decide(int n, int* __restrict__ state, const unsigned long long* __restrict__ M2,
                             int* __restrict__ undecided) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  if (state[I] != ST_UND) return;
  const unsigned long long me = mis_key(ST_UND, I);
  if (M2[I] == me) state[I] = ST_IN;
  else if ((int)(M2[I] >> 62) == ST_IN) state[I] = ST_OUT;
  else atomicAdd(undecided, 1);
}

__global__ void k_root_flags(int n, const int* __restrict__ state, int* __restrict__ flag) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I < n) flag[I] = state[I] == ST_IN;
}

// pass 1: roots keep their id; neighbours join the most strongly connected root
__global__ void k_agg_pass1(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const uint8_t* __restrict__ strong, const double* __restrict__ snorm,
                            const int* __restrict__ state, const uint8_t* __restrict__ iso,
                            const int* __restrict__ rootid, int* __restrict__ agg1) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  if (iso[I]) {
    agg1[I] = -1;
    return;
  }
  if (state[I] == ST_IN) {
    agg1[I] = rootid[I];
    return;
  }
  int best = -1;
  double bs = -1.0;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    if (!strong[k]) continue;
    const int J = col[k];
    if (state[J] != ST_IN) continue;
    if (snorm[k] > bs || (snorm[k] == bs && J < best)) {
      bs = snorm[k];
      best = J;
    }
  }
  agg1[I] = best >= 0 ? rootid[best] : -2;
}

// pass 2: the rest join the aggregate of their most strongly connected assigned neighbour
__global__ void k_agg_pass2(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const uint8_t* __restrict__ strong, const double* __restrict__ snorm,
                            const int* __restrict__ agg1, int* __restrict__ agg) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const int a = agg1[I];
  if (a != -2) {
    agg[I] = a;
    return;
  }
  int best = -1, ba = -1;
  double bs = -1.0;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    if (!strong[k]) continue;
    const int J = col[k];
    const int aj = agg1[J];
    if (aj < 0) continue;
    if (snorm[k] > bs || (snorm[k] == bs && J < best)) {
      bs = snorm[k];
      best = J;
      ba = aj;
    }
  }
  agg[I] = ba;   // -1 (isolated) if nothing was found
}

__global__ void k_count_members(int n, const int* __restrict__ agg, int* __restrict__ cnt) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  if (agg[I] >= 0) atomicAdd(&cnt[agg[I]], 1);
}

__global__ void k_fill_members(int n, const int* __restrict__ agg, const int* __restrict__ off,
                               int* __restrict__ cursor, int* __restrict__ members) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const int a = agg[I];
  if (a < 0) return;
  const int p = atomicAdd(&cursor[a], 1);
  members[off[a] + p] = I;
}

__global__ void k_sort_segments(int nseg, const int* __restrict__ off, int* __restrict__ key,
                                int* __restrict__ aux) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nseg) return;
  const int lo = off[a], hi = off[a + 1];
  for (int i = lo + 1; i < hi; ++i) {
    const int k = key[i];
    const int x = aux ? aux[i] : 0;
    int j = i - 1;
    while (j >= lo && key[j] > k) {
      key[j + 1] = key[j];
      if (aux) aux[j + 1] = aux[j];
      --j;
    }
    key[j + 1] = k;
    if (aux) aux[j + 1] = x;
  }
}

// Tentative prolongator: per aggregate, QR of the near-null space rows.
// Q -> Qn[I][r][j] (node-blocked, br x nns), R -> Bc (column-major, ld = nagg*nns)
__global__ void k_tentative(int nagg, int br, int nns, const int* __restrict__ off,
                            const int* __restrict__ members, const double* __restrict__ B,
                            int64_t ldB, double* __restrict__ Qn, double* __restrict__ Bc,
                            int64_t ldc) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nagg) return;
  const int lo = off[a], hi = off[a + 1];
  // copy B rows into Q storage
  for (int t = lo; t < hi; ++t) {
    const int I = members[t];
    for (int r = 0; r < br; ++r)
      for (int j = 0; j < nns; ++j)
        Qn[((int64_t)I * br + r) * nns + j] = B[(int64_t)j * ldB + (int64_t)I * br + r];
  }
  double R[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) R[i][j] = 0.0;
  for (int j = 0; j < nns; ++j) {
    double n0 = 0.0;
    for (int t = lo; t < hi; ++t)
      for (int r = 0; r < br; ++r) {
        const double v = Qn[((int64_t)members[t] * br + r) * nns + j];
        n0 += v * v;
      }
    n0 = sqrt(n0);
    for (int pass = 0; pass < 2; ++pass) {
      for (int k = 0; k < j; ++k) {
        double dot = 0.0;
        for (int t = lo; t < hi; ++t)
          for (int r = 0; r < br; ++r) {
            const double* q = Qn + ((int64_t)members[t] * br + r) * nns;
            dot += q[k] * q[j];
          }
        R[k][j] += dot;
        for (int t = lo; t < hi; ++t)
          for (int r = 0; r < br; ++r) {
            double* q = Qn + ((int64_t)members[t] * br + r) * nns;
            q[j] -= dot * q[k];
          }
      }
    }
    double nj = 0.0;
    for (int t = lo; t < hi; ++t)
      for (int r = 0; r < br; ++r) {
        const double v = Qn[((int64_t)members[t] * br + r) * nns + j];
        nj += v * v;
      }
    nj = sqrt(nj);
    const bool dead = !(nj > 1e-10 * n0) || n0 == 0.0;
    R[j][j] = dead ? 0.0 : nj;
    const double sc = dead ? 0.0 : 1.0 / nj;
    for (int t = lo; t < hi; ++t)
      for (int r = 0; r < br; ++r) Qn[((int64_t)members[t] * br + r) * nns + j] *= sc;
    if (dead)
      for (int k = 0; k < j; ++k) R[k][j] = 0.0;
  }
  for (int k = 0; k < nns; ++k)
    for (int j = 0; j < nns; ++j) Bc[(int64_t)j * ldc + (int64_t)a * nns + k] = R[k][j];
}

__global__ void k_zero_rows(int n, int stride, const int* __restrict__ agg, double* __restrict__ Qn) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n || agg[I] >= 0) return;
  for (int e = 0; e < stride; ++e) Qn[(int64_t)I * stride + e] = 0.0;
}

// insert c into the sorted list u[0..*len) if absent; false on overflow
__device__ __forceinline__ bool insert_unique(int* u, int& len, int c) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (u[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  if (lo < len && u[lo] == c) return true;
  if (len >= CAP) return false;
  for (int j = len; j > lo; --j) u[j] = u[j - 1];
  u[lo] = c;
  ++len;
  return true;
}

// P = (I - omega D^-1 A) P_tent: count unique aggregate columns per row
__global__ void k_P_count(int n, const int* __restrict__ rp, const int* __restrict__ col,
                          const uint8_t* __restrict__ strong, const int* __restrict__ agg,
                          int* __restrict__ cnt, int* __restrict__ err) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int u[CAP];
  int len = 0;
  bool ok = true;
  if (agg[I] >= 0) ok &= insert_unique(u, len, agg[I]);
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    if (J != I && strong[k] && agg[J] >= 0) ok &= insert_unique(u, len, agg[J]);
  }
  if (!ok) atomicExch(err, 2);
  cnt[I] = len;
}

__global__ void k_P_fill(int n, int br, int nns, const int* __restrict__ rp,
                         const int* __restrict__ col, const double* __restrict__ val,
                         const uint8_t* __restrict__ strong, const int* __restrict__ agg,
                         const double* __restrict__ Qn, const double* __restrict__ dinv,
                         double omega, const int* __restrict__ prp, int* __restrict__ pcol,
                         double* __restrict__ pval) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int u[CAP];
  int len = 0;
  if (agg[I] >= 0) insert_unique(u, len, agg[I]);
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    if (J != I && strong[k] && agg[J] >= 0) insert_unique(u, len, agg[J]);
  }
  const int base = prp[I];
  const int bs = br * nns;
  for (int p = 0; p < len; ++p) {
    pcol[base + p] = u[p];
    double* dst = pval + (int64_t)(base + p) * bs;
    for (int e = 0; e < bs; ++e) dst[e] = 0.0;
  }
  if (agg[I] < 0) return;   // isolated rows keep a zero prolongator row
  const int pI = find_col(pcol, base, base + len, agg[I]);
  if (pI < 0) return;       // capacity overflow, reported by k_P_count
  {
    double* dst = pval + (int64_t)pI * bs;
    for (int e = 0; e < bs; ++e) dst[e] = Qn[(int64_t)I * bs + e];
  }
  // filtered operator: weak off-diagonal blocks are lumped into the diagonal
  // block (row sums, hence the translations, are kept)
  double L[36];
  for (int e = 0; e < br * br; ++e) L[e] = 0.0;
  int kd = -1;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    if (J == I) kd = k;
    if (J == I || !strong[k]) {
      const double* Ablk = val + (int64_t)k * br * br;
      for (int e = 0; e < br * br; ++e) L[e] += Ablk[e];
    }
  }
  if (kd < 0) return;
  double dF[6];
  for (int r = 0; r < br; ++r) {
    const double aii = val[(int64_t)kd * br * br + r * br + r];
    dF[r] = L[r * br + r] > 0.1 * aii ? 1.0 / L[r * br + r] : dinv[(int64_t)I * br + r];
  }
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    const bool diag = J == I;
    if (!diag && !strong[k]) continue;
    const int a = agg[J];
    if (a < 0) continue;
    const int p = diag ? pI : find_col(pcol, base, base + len, a);
    if (p < 0) continue;
    double* dst = pval + (int64_t)p * bs;
    const double* Ablk = diag ? L : val + (int64_t)k * br * br;
    const double* Q = Qn + (int64_t)J * bs;
    for (int r = 0; r < br; ++r) {
      const double w = omega * dF[r];
      for (int j = 0; j < nns; ++j) {
        double s = 0.0;
        for (int c = 0; c < br; ++c) s += Ablk[r * br + c] * Q[c * nns + j];
        dst[r * nns + j] -= w * s;
      }
    }
  }
}

// transpose: count entries per column
__global__ void k_T_count(int n, const int* __restrict__ rp, const int* __restrict__ col,
                          int* __restrict__ cnt) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  for (int k = rp[I]; k < rp[I + 1]; ++k) atomicAdd(&cnt[col[k]], 1);
}

__global__ void k_T_fill(int n, const int* __restrict__ rp, const int* __restrict__ col,
                         const int* __restrict__ trp, int* __restrict__ cursor,
                         int* __restrict__ tcol, int* __restrict__ src) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int c = col[k];
    const int p = trp[c] + atomicAdd(&cursor[c], 1);
    tcol[p] = I;
    src[p] = k;
  }
}

__global__ void k_T_vals(int64_t nnz, int br, int bc, const int* __restrict__ src,
                         const double* __restrict__ val, double* __restrict__ tval) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  const double* s = val + (int64_t)src[p] * br * bc;   // br x bc
  double* d = tval + p * bc * br;                       // bc x br
  for (int r = 0; r < br; ++r)
    for (int c = 0; c < bc; ++c) d[c * br + r] = s[r * bc + c];
}

// C = X Y, row-wise with sorted unique columns
__global__ void k_mm_count(int n, const int* __restrict__ xrp, const int* __restrict__ xcol,
                           const int* __restrict__ yrp, const int* __restrict__ ycol,
                           int* __restrict__ cnt, int* __restrict__ err) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int u[CAP];
  int len = 0;
  bool ok = true;
  for (int k = xrp[I]; k < xrp[I + 1]; ++k) {
    const int K = xcol[k];
    for (int l = yrp[K]; l < yrp[K + 1]; ++l) ok &= insert_unique(u, len, ycol[l]);
  }
  if (!ok) atomicExch(err, 3);
  cnt[I] = len;
}

__global__ void k_mm_fill(int n, int xr, int xc, int yc, const int* __restrict__ xrp,
                          const int* __restrict__ xcol, const double* __restrict__ xval,
                          const int* __restrict__ yrp, const int* __restrict__ ycol,
                          const double* __restrict__ yval, const int* __restrict__ crp,
                          int* __restrict__ ccol, double* __restrict__ cval) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  int u[CAP];
  int len = 0;
  for (int k = xrp[I]; k < xrp[I + 1]; ++k) {
    const int K = xcol[k];
    for (int l = yrp[K]; l < yrp[K + 1]; ++l) insert_unique(u, len, ycol[l]);
  }
  const int base = crp[I];
  const int bs = xr * yc;
  for (int p = 0; p < len; ++p) {
    ccol[base + p] = u[p];
    for (int e = 0; e < bs; ++e) cval[(int64_t)(base + p) * bs + e] = 0.0;
  }
  for (int k = xrp[I]; k < xrp[I + 1]; ++k) {
    const int K = xcol[k];
    const double* X = xval + (int64_t)k * xr * xc;
    for (int l = yrp[K]; l < yrp[K + 1]; ++l) {
      const int p = find_col(ccol, base, base + len, ycol[l]);
      if (p < 0) continue;   // capacity overflow, reported by k_mm_count
      const double* Y = yval + (int64_t)l * xc * yc;
      double* C = cval + (int64_t)p * bs;
      for (int r = 0; r < xr; ++r)
        for (int c = 0; c < yc; ++c) {
          double s = 0.0;
          for (int m = 0; m < xc; ++m) s += X[r * xc + m] * Y[m * yc + c];
          C[r * yc + c] += s;
        }
    }
  }
}

// ---- warp-per-row SpGEMM C = X Y (set-up Galerkin products) ---------------
// One warp per row of X.  Symbolic: the candidate columns (columns of the Y
// rows named by the row of X) go into a shared-memory hash set, which keeps
// each column once whatever the insertion order.  Numeric: the unique columns
// are compacted, sorted (bitonic, in shared memory) and written, and the block
// products are added into the output row in the fixed order of the row of X
// and the rows of Y, lanes splitting each block -- no atomics on values, so
// the result is deterministic.  A row with more than MM_HS/2 unique columns
// sets *overflow (the caller then uses the row-per-thread kernels).
constexpr int MM_WS = 4;      // warps per block
constexpr int MM_HS = 1024;   // hash slots per warp (rows of up to 512 unique columns; the
                              // 3d hierarchies stay below, and wider tables cost occupancy)

__device__ __forceinline__ int mm_insert(int* h, int c, bool* full) {
  unsigned slot = ((unsigned)c * 2654435761u) & (MM_HS - 1);
  for (int t = 0; t < MM_HS; ++t) {
    const int old = atomicCAS(&h[slot], -1, c);
    if (old == -1) return 1;
    if (old == c) return 0;
    slot = (slot + 1) & (MM_HS - 1);
  }
  *full = true;
  return 0;
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// fill h (cleared by the caller) with the columns of row I of X Y; returns the count
__device__ int mm_gather(int I, const int* __restrict__ xrp, const int* __restrict__ xcol,
                         const int* __restrict__ yrp, const int* __restrict__ ycol, int* h,
                         bool* full) {
  const int lane = threadIdx.x & 31;
  int ins = 0;
  for (int k = xrp[I]; k < xrp[I + 1]; ++k) {
    const int K = xcol[k];
    for (int l = yrp[K] + lane; l < yrp[K + 1]; l += 32) ins += mm_insert(h, ycol[l], full);
  }
  __syncwarp();
  return warp_sum_int(ins);
}

__global__ void __launch_bounds__(32 * MM_WS) k_mm_count_w(int n, const int* __restrict__ xrp,
                                                          const int* __restrict__ xcol,
                                                          const int* __restrict__ yrp,
                                                          const int* __restrict__ ycol,
                                                          int* __restrict__ cnt,
                                                          int* __restrict__ overflow) {
  __shared__ int hs[MM_WS][MM_HS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int I = blockIdx.x * MM_WS + w;
  int* h = hs[w];
  for (int e = lane; e < MM_HS; e += 32) h[e] = -1;
  __syncwarp();
  if (I >= n) return;   // the whole warp leaves together
  bool full = false;
  const int c = mm_gather(I, xrp, xcol, yrp, ycol, h, &full);
  const bool bad = __any_sync(0xffffffffu, full) || c > MM_HS / 2;
  if (lane == 0) {
    cnt[I] = c;
    if (bad) atomicExch(overflow, 1);
  }
}

__global__ void __launch_bounds__(32 * MM_WS) k_mm_fill_w(int n, int xr, int xc, int yc,
                                                         const int* __restrict__ xrp,
                                                         const int* __restrict__ xcol,
                                                         const double* __restrict__ xval,
                                                         const int* __restrict__ yrp,
                                                         const int* __restrict__ ycol,
                                                         const double* __restrict__ yval,
                                                         const int* __restrict__ crp,
                                                         int* __restrict__ ccol,
                                                         double* __restrict__ cval) {
  __shared__ int hs[MM_WS][MM_HS];
  __shared__ int ls[MM_WS][MM_HS / 2];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int I = blockIdx.x * MM_WS + w;
  int* h = hs[w];
  int* list = ls[w];
  for (int e = lane; e < MM_HS; e += 32) h[e] = -1;
  __syncwarp();
  if (I >= n) return;
  bool full = false;
  const int cnt = mm_gather(I, xrp, xcol, yrp, ycol, h, &full);   // = crp[I+1] - crp[I]
  // compact the keys, then sort them (padded to a power of two with INT_MAX)
  int m = 1;
  while (m < cnt) m <<= 1;
  int base = 0;
  for (int e0 = 0; e0 < MM_HS; e0 += 32) {
    const int key = h[e0 + lane];
    const unsigned b = __ballot_sync(0xffffffffu, key >= 0);
    if (key >= 0) list[base + __popc(b & ((1u << lane) - 1u))] = key;
    base += __popc(b);
  }
  for (int e = cnt + lane; e < m; e += 32) list[e] = 0x7fffffff;
  __syncwarp();
  for (int k = 2; k <= m; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < m; i += 32) {
        const int p = i ^ j;
        if (p > i) {
          const bool up = (i & k) == 0;
          const int a = list[i], b2 = list[p];
          if ((a > b2) == up) {
            list[i] = b2;
            list[p] = a;
          }
        }
      }
      __syncwarp();
    }
  const int c0 = crp[I];
  const int bs = xr * yc;
  for (int e = lane; e < cnt; e += 32) ccol[c0 + e] = list[e];
  for (int e = lane; e < cnt * bs; e += 32) cval[(int64_t)c0 * bs + e] = 0.0;
  __syncwarp();
  // block products in the fixed order of X's row and Y's rows
  for (int k = xrp[I]; k < xrp[I + 1]; ++k) {
    const int K = xcol[k];
    const double* Xb = xval + (int64_t)k * xr * xc;
    for (int l = yrp[K]; l < yrp[K + 1]; ++l) {
      const int c = ycol[l];
      int lo = 0, hi = cnt;   // every lane finds the same slot
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (list[mid] < c) lo = mid + 1;
        else hi = mid;
      }
      const double* Yb = yval + (int64_t)l * xc * yc;
      double* Cb = cval + (int64_t)(c0 + lo) * bs;
      for (int e = lane; e < bs; e += 32) {
        const int r = e / yc, cc = e - r * yc;
        double s = 0.0;
        for (int q = 0; q < xc; ++q) s += Xb[r * xc + q] * Yb[q * yc + cc];
        Cb[e] += s;
      }
      __syncwarp();
    }
  }
}

// zero diagonal entries (dead coarse DoFs) -> 1
__global__ void k_fix_diag(int n, int b, const int* __restrict__ rp, const int* __restrict__ col,
                           double* __restrict__ val) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  const int k = find_col(col, rp[I], rp[I + 1], I);
  if (k < 0) return;
  double* v = val + (int64_t)k * b * b;
  for (int a = 0; a < b; ++a) {
    bool zero_row = true;
    for (int kk = rp[I]; kk < rp[I + 1] && zero_row; ++kk)
      for (int c = 0; c < b; ++c)
        if (val[(int64_t)kk * b * b + a * b + c] != 0.0) zero_row = false;
    if (zero_row) v[a * b + a] = 1.0;
  }
}

__global__ void k_densify(int n, int b, const int* __restrict__ rp, const int* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ D, int ld) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= n) return;
  for (int k = rp[I]; k < rp[I + 1]; ++k) {
    const int J = col[k];
    for (int r = 0; r < b; ++r)
      for (int c = 0; c < b; ++c)
        D[(int64_t)(I * b + r) * ld + J * b + c] = val[(int64_t)k * b * b + r * b + c];
  }
}

// Gauss-Jordan inverse with partial pivoting, one block (n small)
// Gauss-Jordan with partial pivoting spread over the GPU: per pivot k one
// block chooses the pivot row, swaps it into row k and scales it (k_gj_pivot),
// then one block per row eliminates column k from it (k_gj_elim).
__global__ void k_gj_identity(int n, double* __restrict__ Inv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (int64_t)n * n) Inv[e] = (e / n == e % n) ? 1.0 : 0.0;
}

__global__ void k_gj_pivot(int n, int k, double* __restrict__ A, double* __restrict__ Inv,
                           int* __restrict__ err) {
  __shared__ double pmax[256];
  __shared__ int pidx[256];
  const int t = threadIdx.x;
  double best = -1.0;
  int bi = k;
  for (int r = k + t; r < n; r += blockDim.x) {
    const double v = fabs(A[(int64_t)r * n + k]);
    if (v > best) {
      best = v;
      bi = r;
    }
  }
  pmax[t] = best;
  pidx[t] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {   // max, ties to the lower row
    if (t < o && (pmax[t + o] > pmax[t] || (pmax[t + o] == pmax[t] && pidx[t + o] < pidx[t]))) {
      pmax[t] = pmax[t + o];
      pidx[t] = pidx[t + o];
    }
    __syncthreads();
  }
  const int p = pidx[0];
  if (t == 0 && !(pmax[0] > 0.0)) atomicExch(err, 4);
  if (p != k) {
    for (int c = t; c < n; c += blockDim.x) {
      double x = A[(int64_t)k * n + c];
      A[(int64_t)k * n + c] = A[(int64_t)p * n + c];
      A[(int64_t)p * n + c] = x;
      x = Inv[(int64_t)k * n + c];
      Inv[(int64_t)k * n + c] = Inv[(int64_t)p * n + c];
      Inv[(int64_t)p * n + c] = x;
    }
  }
  __syncthreads();
  const double dk = A[(int64_t)k * n + k];
  const double inv = dk != 0.0 ? 1.0 / dk : 0.0;
  __syncthreads();
  for (int c = t; c < n; c += blockDim.x) {
    A[(int64_t)k * n + c] *= inv;
    Inv[(int64_t)k * n + c] *= inv;
  }
}

// block r != k: row r -= A[r][k] * row k (row k is only read here)
__global__ void k_gj_elim(int n, int k, double* __restrict__ A, double* __restrict__ Inv) {
  const int r = blockIdx.x;
  if (r == k) return;
  const double f = A[(int64_t)r * n + k];
  if (f == 0.0) return;
  for (int c = k + 1 + threadIdx.x; c < n; c += blockDim.x)
    A[(int64_t)r * n + c] -= f * A[(int64_t)k * n + c];
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    Inv[(int64_t)r * n + c] -= f * Inv[(int64_t)k * n + c];
  __syncthreads();
  if (threadIdx.x == 0) A[(int64_t)r * n + k] = 0.0;
}

// Lanczos recurrence on S = D^-1/2 A D^-1/2 with every scalar kept on the device
// (FP64 scalars; vectors in T = double, or float for mixed-precision hierarchies):
// al[j] = <S v_j, v_j>, nb2[j] = ||w_j||^2, beta_j = sqrt(nb2[j])
template <class T>
__global__ void k_lz_sqrt(int64_t n, const T* __restrict__ dinv, T* __restrict__ dh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dh[i] = sqrt(dinv[i]);
}
// w = sg * dh .* y   (sg = -1 when y holds -A x)
template <class T>
__global__ void k_lz_scale(int64_t n, const T* __restrict__ dh, const T* __restrict__ y,
                           T* __restrict__ w, T sg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = sg * (dh[i] * y[i]);
}
// w -= al[j] v + beta_{j-1} vp   (no vp term at j = 0)
template <class T>
__global__ void k_lz_orth(int64_t n, T* __restrict__ w, const T* __restrict__ v,
                          const T* __restrict__ vp, const double* __restrict__ al,
                          const double* __restrict__ nb2, int j) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T a = (T)al[j];
  const T beta = j > 0 ? (T)sqrt(fmax(nb2[j - 1], 0.0)) : T(0);
  w[i] -= a * v[i] + (j > 0 ? beta * vp[i] : T(0));
}
// v_next = w / ||w|| (0 after a breakdown), t = dh .* v_next
template <class T>
__global__ void k_lz_next(int64_t n, const T* __restrict__ w, const double* __restrict__ nb2,
                          int j, const T* __restrict__ dh, T* __restrict__ vn, T* __restrict__ t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T q = nb2[j] > 0.0 ? (T)(1.0 / sqrt(nb2[j])) : T(0);
  const T x = w[i] * q;
  vn[i] = x;
  t[i] = dh[i] * x;
}

template <class T>
__global__ void k_hash_vec(int64_t n, T* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (T)((double)(hash32((uint32_t)i * 2654435761u + 12345u) & 0xffffff) / 16777216.0 + 0.1);
}

__global__ void k_to_float(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// --------------------------------------------------------------- V-cycle ---
template <class T>
__global__ void k_dense_mv(int n, const T* __restrict__ M, const T* __restrict__ x, T* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  T s = 0;
  for (int c = lane; c < n; c += 32) s += M[(int64_t)row * n + c] * x[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

template <class Tin, class Tout>
__global__ void k_convert(int64_t n, const Tin* __restrict__ a, Tout* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (Tout)a[i];
}

template <class T>
const T* dinvs(const AmgLevel& L);
template <>
const double* dinvs<double>(const AmgLevel& L) { return L.dinv; }
template <>
const float* dinvs<float>(const AmgLevel& L) { return L.dinvf; }

template <class T>
void spmv_t(const Bsr& A, const T* x, T* y, T alpha, T beta, cudaStream_t s);
template <>
void spmv_t<double>(const Bsr& A, const double* x, double* y, double a, double b, cudaStream_t s) {
  bsr_spmv(A, x, y, a, b, s);
}
template <>
void spmv_t<float>(const Bsr& A, const float* x, float* y, float a, float b, cudaStream_t s) {
  bsr_spmv_f(A, x, y, a, b, s);
}

template <class T>
const T* stencil_vals(const AmgLevel& L);
template <>
const double* stencil_vals<double>(const AmgLevel& L) { return L.st; }
template <>
const float* stencil_vals<float>(const AmgLevel& L) { return L.stf; }

template <class T>
void vcycle_level(Amg& amg, int l, const T* rhs, T* x, cudaStream_t s,
                  const double* rhs64 = nullptr, double* out64 = nullptr);

// Levels 1.. of the cycle (many small, launch-bound kernels) replayed as one
// CUDA graph.  It is captured on first use after each build, on a private
// stream, and launched on the caller's stream; if capture is not possible the
// levels run as ordinary launches.
template <class T>
void coarse_cycle(Amg& amg, T* cb, T* cx, cudaStream_t s) {
  if (!amg.graph && amg.use_graph) {
    bool ok = true;
    if (!amg.cap_stream) ok = cudaStreamCreateWithFlags(&amg.cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCapture(amg.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      set_capturing(true);
      try {
        vcycle_level<T>(amg, 1, cb, cx, amg.cap_stream);
      } catch (...) {
        ok = false;
      }
      amg.graph_bytes = captured_bytes();
      set_capturing(false);
      cudaGraph_t g = nullptr;
      if (cudaStreamEndCapture(amg.cap_stream, &g) != cudaSuccess) ok = false;
      if (ok && g) {
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        int kern = 0;
        for (auto nd : nodes) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
        }
        amg.graph_kernels = kern;
        if (cudaGraphInstantiate(&amg.graph, g, 0) != cudaSuccess) {
          amg.graph = nullptr;
          ok = false;
        }
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    if (!ok) amg.use_graph = false;
  }
  if (amg.graph) {
    ProfScope ps(amg.lev[0].A.br > 1 ? "coarse_levels_graph_u" : "coarse_levels_graph_phi",
                 amg.graph_bytes, s, amg.graph_kernels);
    PFF_CUDA(cudaGraphLaunch(amg.graph, s));
  } else {
    vcycle_level<T>(amg, 1, cb, cx, s);
  }
}

// rhs64 (stencil levels only): the first step reads the FP64 right-hand side and
// stores it into rhs; out64: the last step writes the result there in FP64
// (x is then not written)
template <class T>
void smooth(const AmgLevel& L, int degree, double ratio, const T* rhs, T* x, T* t, T* d, bool zero_start,
            cudaStream_t s, const double* rhs64 = nullptr, T* rhs_store = nullptr,
            double* out64 = nullptr) {
  // Chebyshev iteration for D^-1 A on [lmax/30, 1.1 lmax]
  const double beta = 1.1 * L.lmax, alpha = L.lmax / ratio;
  const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const Bsr& A = L.A;
  const int nb = A.nrows, b = A.br;
  if ((rhs64 || out64) && !L.stencil) fail(PFF_ERR_INVALID_ARG, "FP64 cycle ends need a stencil level");
  T* cur = x;
  T* nxt = t;
  // first step: d = r / theta
  if (L.stencil) {
    launch_stencil_cheb<T>(L.mesh, nb, b, stencil_vals<T>(L), dinvs<T>(L), rhs, cur, nxt, d, 0.0,
                           1.0 / theta, zero_start ? 1 : 0, s, sizeof(T) == 4 && L.stf_node_major,
                           rhs64, rhs_store, degree == 1 ? out64 : nullptr);
  } else {
    bsr_cheb<T>(A, dinvs<T>(L), rhs, cur, nxt, d, T(0), T(1.0 / theta), zero_start, s);
  }
  std::swap(cur, nxt);
  for (int k = 1; k < degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    if (L.stencil) {
      launch_stencil_cheb<T>(L.mesh, nb, b, stencil_vals<T>(L), dinvs<T>(L), rhs, cur, nxt, d,
                             rn * rho, 2.0 * rn / delta, 0, s, sizeof(T) == 4 && L.stf_node_major,
                             nullptr, nullptr, k == degree - 1 ? out64 : nullptr);
    } else {
      bsr_cheb<T>(A, dinvs<T>(L), rhs, cur, nxt, d, T(rn * rho), T(2.0 * rn / delta), false, s);
    }
    std::swap(cur, nxt);
    rho = rn;
  }
  if (cur != x && !out64)
    PFF_CUDA(cudaMemcpyAsync(x, cur, sizeof(T) * (size_t)nb * b, cudaMemcpyDeviceToDevice, s));
  PFF_LAUNCH("chebyshev");
}

// rhs64 / out64 (level 0 of a mixed cycle on a stencil level): the FP64 input
// and output of the cycle, converted inside the first and last smoothing steps;
// rhs then names the level's own FP32 right-hand side buffer, filled there.
template <class T>
void vcycle_level(Amg& amg, int l, const T* rhs, T* x, cudaStream_t s, const double* rhs64,
                  double* out64) {
  if (l == (int)amg.lev.size()) {
    const T* M = nullptr;
    if constexpr (sizeof(T) == 8) M = reinterpret_cast<const T*>(amg.cinv);
    else M = reinterpret_cast<const T*>(amg.cinvf);
    ProfScope ps("coarse_solve", (double)sizeof(T) * amg.nc * (amg.nc + 2.0), s);
    k_dense_mv<T><<<grid_for(amg.nc, 8), 256, 0, s>>>(amg.nc, M, rhs, x);
    PFF_LAUNCH("coarse");
    return;
  }
  AmgLevel& L = amg.lev[l];
  T* t = reinterpret_cast<T*>(L.t);
  T* d = reinterpret_cast<T*>(L.d);
  T* r = reinterpret_cast<T*>(L.r);
  const int deg = l == 0 ? amg.cheb_degree : amg.cheb_degree_coarse;
  T* rhs_store = rhs64 ? const_cast<T*>(rhs) : nullptr;
  smooth<T>(L, deg, amg.cheb_ratio, rhs, x, t, d, true, s, rhs64, rhs_store);
  if (L.terminal) {
    smooth<T>(L, deg, amg.cheb_ratio, rhs, x, t, d, false, s, nullptr, nullptr, out64);
    return;
  }
  const Bsr& A = L.A;
  if (L.stencil) {
    launch_stencil_resid<T>(L.mesh, A.nrows, A.br, stencil_vals<T>(L), rhs, x, r, s,
                            sizeof(T) == 4 && L.stf_node_major);
  } else {
    bsr_resid<T>(A, rhs, x, r, s);
  }
  const bool last = l + 1 == (int)amg.lev.size();
  T* cb = last ? reinterpret_cast<T*>(amg.cb) : reinterpret_cast<T*>(amg.lev[l + 1].b);
  T* cx = last ? reinterpret_cast<T*>(amg.cx) : reinterpret_cast<T*>(amg.lev[l + 1].x);
  spmv_t<T>(L.R, r, cb, T(1), T(0), s);
  if (l == 0 && amg.use_graph && !amg.inline_levels) coarse_cycle<T>(amg, cb, cx, s);
  else vcycle_level<T>(amg, l + 1, cb, cx, s);
  spmv_t<T>(L.P, cx, x, T(1), T(1), s);
  smooth<T>(L, deg, amg.cheb_ratio, rhs, x, t, d, false, s, nullptr, nullptr, out64);
}

struct SetupScratch {
  int* err = nullptr;
  int* h_err = nullptr;
  double* red = nullptr;
  double* h_red = nullptr;
};

// largest eigenvalue of the symmetric tridiagonal matrix (alpha, beta) by bisection
// on the Sturm sequence count
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {   // number of eigenvalues < x
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      q = a[i] - x - (i > 0 ? bb / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-12 * std::max(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) < m) lo = mid;
    else hi = mid;
  }
  return hi;
}

// lambda_max(D^-1 A) by Lanczos on the similar symmetric matrix D^-1/2 A D^-1/2:
// the extreme Ritz value converges from below much faster than power iteration
// on the clustered spectra of graded meshes.
void lz_dot(const double* x, const double* y, int64_t n, double* out, double* partials,
            cudaStream_t s) {
  dot_dev(x, y, n, out, partials, s);
}
void lz_dot(const float* x, const float* y, int64_t n, double* out, double* partials,
            cudaStream_t s) {
  dot_dev_f32(x, y, n, out, partials, s);
}
void lz_spmv(const Bsr& A, const double* x, double* y, cudaStream_t s) { bsr_spmv(A, x, y, 1.0, 0.0, s); }
void lz_spmv(const Bsr& A, const float* x, float* y, cudaStream_t s) { bsr_spmv_f(A, x, y, 1.f, 0.f, s); }

// The operator of the Lanczos recurrence: the level's BSR copy, or at the
// finest level the node stencil itself (the smoother's own operator; for the
// 27-slot 3d stencils about 4x faster than the BSR copy, whose rows the
// sparse-kernel tuner never times because the V-cycle does not use them).
template <class T>
struct LzOperator {
  const Bsr* A = nullptr;
  const AmgParams* st = nullptr;   // non-null: apply st's stencil
  T* zero = nullptr;               // zero right-hand side of the stencil residual kernel
};

template <class T>
const T* lz_stencil_vals(const AmgParams& p);
template <>
const double* lz_stencil_vals<double>(const AmgParams& p) { return p.st; }
template <>
const float* lz_stencil_vals<float>(const AmgParams& p) { return p.stf; }

// y = A x, or y = -A x (returns -1) through the stencil residual with a zero rhs
template <class T>
T lz_apply(const LzOperator<T>& op, const T* x, T* y, cudaStream_t s) {
  if (!op.st) {
    lz_spmv(*op.A, x, y, s);
    return T(1);
  }
  launch_stencil_resid<T>(op.st->mesh, op.A->nrows, op.A->br, lz_stencil_vals<T>(*op.st), op.zero, x,
                          y, s, sizeof(T) == 4 && op.st->stf_node_major);
  return T(-1);
}

// T = float runs the recurrence on the FP32 copy of A (A.valf) or of the
// stencil: the estimate only sets the Chebyshev interval and the prolongator
// damping
template <class T>
double estimate_lmax(const Bsr& A, const T* dinv, cudaStream_t s, double* partials,
                     double* dred, double* hred, const AmgParams* stencil = nullptr) {
  (void)hred;
  const int64_t n = (int64_t)A.nrows * A.br;
  LzOperator<T> op;
  op.A = &A;
  if (stencil && lz_stencil_vals<T>(*stencil)) {
    op.st = stencil;
    op.zero = dalloc<T>(n);
    PFF_CUDA(cudaMemsetAsync(op.zero, 0, sizeof(T) * n, s));
  }
  const int steps = (int)std::min<int64_t>(30, n);
  const unsigned g = grid_for(n, 256);
  T* v = dalloc<T>(n);
  T* vp = dalloc<T>(n);
  T* w = dalloc<T>(n);
  T* t = dalloc<T>(n);
  T* y = dalloc<T>(n);
  T* dh = dalloc<T>(n);
  double* al = dalloc<double>(2 * steps);
  double* nb2 = al + steps;
  PFF_CUDA(cudaMemsetAsync(vp, 0, sizeof(T) * n, s));
  count_launch(3);
  k_lz_sqrt<T><<<g, 256, 0, s>>>(n, dinv, dh);
  k_hash_vec<T><<<g, 256, 0, s>>>(n, w);
  lz_dot(w, w, n, dred, partials, s);
  k_lz_next<T><<<g, 256, 0, s>>>(n, w, dred, 0, dh, v, t);   // v_0 = w / ||w||, t = dh .* v_0
  // largest Ritz value of T_m (m = done steps) up to the first breakdown
  // (beta_j ~ 0: an invariant subspace was found); *broke tells whether it did
  std::vector<double> h(2 * steps);
  auto ritz = [&](int done, bool* broke) {
    PFF_CUDA(cudaMemcpyAsync(h.data(), al, sizeof(double) * steps, cudaMemcpyDeviceToHost, s));
    PFF_CUDA(cudaMemcpyAsync(h.data() + steps, nb2, sizeof(double) * steps, cudaMemcpyDeviceToHost, s));
    PFF_CUDA(cudaStreamSynchronize(s));
    std::vector<double> a, b;
    *broke = false;
    for (int j = 0; j < done; ++j) {
      a.push_back(h[j]);
      const double bn = std::sqrt(std::max(h[steps + j], 0.0));
      if (!(bn > 1e-14 * std::fabs(h[j]))) {
        *broke = true;
        break;
      }
      if (j + 1 == done) break;
      b.push_back(bn);
    }
    return a.empty() ? 1.0 : tridiag_max_eig(a, b);
  };
  // checkpoints: stop once the largest Ritz value moved by less than 1e-3
  // relative over the last 6 steps (it increases monotonically toward lmax)
  double lam = 0.0, prev = -1.0;
  for (int j = 0; j < steps; ++j) {
    const T sg = lz_apply(op, t, y, s);                       // y = sg A D^-1/2 v_j
    count_launch(3);
    k_lz_scale<T><<<g, 256, 0, s>>>(n, dh, y, w, sg);         // w = S v_j
    lz_dot(w, v, n, al + j, partials, s);
    k_lz_orth<T><<<g, 256, 0, s>>>(n, w, v, vp, al, nb2, j);
    lz_dot(w, w, n, nb2 + j, partials, s);
    k_lz_next<T><<<g, 256, 0, s>>>(n, w, nb2, j, dh, vp, t);  // v_{j+1} into the v_{j-1} buffer
    std::swap(v, vp);
    const int done = j + 1;
    if (done == steps || (done >= 12 && done % 6 == 0)) {
      bool broke = false;
      lam = ritz(done, &broke);
      if (broke || done == steps || (prev > 0.0 && lam - prev <= 1e-3 * lam)) break;
      prev = lam;
    }
  }
  PFF_LAUNCH("lmax");
  dfree(op.zero);
  dfree(v);
  dfree(vp);
  dfree(w);
  dfree(t);
  dfree(y);
  dfree(dh);
  dfree(al);
  return std::isfinite(lam) && lam > 0.0 ? lam : 1.0;
}

// C = X * Y (BSR)
void spgemm(const Bsr& X, const Bsr& Y, Bsr& C, int* err, cudaStream_t s) {
  C.nrows = X.nrows;
  C.ncols = Y.ncols;
  C.br = X.br;
  C.bc = Y.bc;
  C.rowptr = dalloc<int>(X.nrows + 1);
  int* cnt = dalloc<int>(X.nrows + 2);
  int* overflow = cnt + X.nrows + 1;
  PFF_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int), s));
  // warp-per-row kernels first; rows wider than their shared tables fall back
  const unsigned gw = (unsigned)((X.nrows + MM_WS - 1) / MM_WS);
  count_launch();
  k_mm_count_w<<<gw, 32 * MM_WS, 0, s>>>(X.nrows, X.rowptr, X.col, Y.rowptr, Y.col, cnt, overflow);
  PFF_LAUNCH("mm_count_w");
  int h_over = 0;
  PFF_CUDA(cudaMemcpyAsync(&h_over, overflow, sizeof(int), cudaMemcpyDeviceToHost, s));
  PFF_CUDA(cudaStreamSynchronize(s));
  const unsigned g = grid_for(X.nrows, 128);
  if (h_over && verbose())
    std::fprintf(stderr, "[pff] SpGEMM %d rows: a row exceeds %d columns, row-per-thread kernels\n",
                 X.nrows, MM_HS / 2);
  if (h_over) {
    count_launch();
    k_mm_count<<<g, 128, 0, s>>>(X.nrows, X.rowptr, X.col, Y.rowptr, Y.col, cnt, err);
    PFF_LAUNCH("mm_count");
  }
  int total = 0;
  exclusive_scan_int(cnt, C.rowptr, X.nrows, &total, s);
  C.nnzb = total;
  C.col = dalloc<int>(total);
  C.val = dalloc<double>((size_t)total * C.br * C.bc);
  count_launch();
  if (h_over) {
    k_mm_fill<<<g, 128, 0, s>>>(X.nrows, X.br, X.bc, Y.bc, X.rowptr, X.col, X.val, Y.rowptr,
                                Y.col, Y.val, C.rowptr, C.col, C.val);
  } else {
    k_mm_fill_w<<<gw, 32 * MM_WS, 0, s>>>(X.nrows, X.br, X.bc, Y.bc, X.rowptr, X.col, X.val,
                                          Y.rowptr, Y.col, Y.val, C.rowptr, C.col, C.val);
  }
  PFF_LAUNCH("mm_fill");
  dfree(cnt);
}

void transpose(const Bsr& P, Bsr& R, cudaStream_t s) {
  R.nrows = P.ncols;
  R.ncols = P.nrows;
  R.br = P.bc;
  R.bc = P.br;
  R.nnzb = P.nnzb;
  R.rowptr = dalloc<int>(R.nrows + 1);
  int* cnt = dalloc<int>(R.nrows + 1);
  int* cursor = dalloc<int>(R.nrows + 1);
  PFF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (R.nrows + 1), s));
  PFF_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * (R.nrows + 1), s));
  count_launch();
  k_T_count<<<grid_for(P.nrows, 256), 256, 0, s>>>(P.nrows, P.rowptr, P.col, cnt);
  int total = 0;
  exclusive_scan_int(cnt, R.rowptr, R.nrows, &total, s);
  R.col = dalloc<int>(total);
  int* src = dalloc<int>(total);
  count_launch();
  k_T_fill<<<grid_for(P.nrows, 256), 256, 0, s>>>(P.nrows, P.rowptr, P.col, R.rowptr, cursor,
                                                  R.col, src);
  count_launch();
  k_sort_segments<<<grid_for(R.nrows, 128), 128, 0, s>>>(R.nrows, R.rowptr, R.col, src);
  R.val = dalloc<double>((size_t)total * R.br * R.bc);
  count_launch();
  k_T_vals<<<grid_for(total, 256), 256, 0, s>>>(total, P.br, P.bc, src, P.val, R.val);
  PFF_LAUNCH("transpose");
  PFF_CUDA(cudaStreamSynchronize(s));
  dfree(cnt);
  dfree(cursor);
  dfree(src);
}

void copy_bsr(const Bsr& A, Bsr& C, cudaStream_t s) {
  C.nrows = A.nrows;
  C.ncols = A.ncols;
  C.br = A.br;
  C.bc = A.bc;
  C.nnzb = A.nnzb;
  C.rowptr = dalloc<int>(A.nrows + 1);
  C.col = dalloc<int>(A.nnzb);
  C.val = dalloc<double>((size_t)A.nnzb * A.br * A.bc);
  PFF_CUDA(cudaMemcpyAsync(C.rowptr, A.rowptr, sizeof(int) * (A.nrows + 1), cudaMemcpyDeviceToDevice, s));
  PFF_CUDA(cudaMemcpyAsync(C.col, A.col, sizeof(int) * A.nnzb, cudaMemcpyDeviceToDevice, s));
  PFF_CUDA(cudaMemcpyAsync(C.val, A.val, sizeof(double) * A.nnzb * A.br * A.bc,
                           cudaMemcpyDeviceToDevice, s));
}

void make_float(Bsr& A, cudaStream_t s) {
  const int64_t nv = A.nnzb * A.br * A.bc;
  A.valf = dalloc<float>(nv);
  count_launch();
  k_to_float<<<grid_for(nv, 256), 256, 0, s>>>(nv, A.val, A.valf);
  PFF_LAUNCH("to_float");
}

void check_err(SetupScratch& sc, cudaStream_t s, const char* where) {
  PFF_CUDA(cudaMemcpyAsync(sc.h_err, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PFF_CUDA(cudaStreamSynchronize(s));
  if (*sc.h_err) fail(PFF_ERR_CAPACITY, std::string("AMG setup failed in ") + where + " (code " +
                                           std::to_string(*sc.h_err) + ")");
}

}  // namespace

void Amg::release() {
  if (graph) cudaGraphExecDestroy(graph);
  graph = nullptr;
  graph_kernels = 0;
  if (cap_stream) cudaStreamDestroy(cap_stream);
  cap_stream = nullptr;
  for (auto& L : lev) {
    L.A.release();
    L.P.release();
    L.R.release();
    dfree(L.dinv);
    dfree(L.dinvf);
    dfree(L.x);
    dfree(L.b);
    dfree(L.r);
    dfree(L.d);
    dfree(L.t);
  }
  lev.clear();
  dfree(cinv);
  dfree(cinvf);
  dfree(cx);
  dfree(cb);
  cinv = nullptr;
  cinvf = nullptr;
  cx = cb = nullptr;
  built = 0;
}

// lambda_max of D^-1 A for a level; mixed hierarchies first make the level's
// FP32 copies (A.valf, dinvf), which the FP32 V-cycle needs anyway
// stencil: the finest level's node stencil (null on coarser levels or when none is given)
double level_lmax(Amg& amg, AmgLevel& L, cudaStream_t s, double* partials, SetupScratch& sc,
                  const AmgParams* stencil) {
  if (!amg.mixed) return estimate_lmax<double>(L.A, L.dinv, s, partials, sc.red, sc.h_red, stencil);
  const int64_t n = (int64_t)L.A.nrows * L.A.br;
  make_float(L.A, s);
  L.dinvf = dalloc<float>(n);
  count_launch();
  k_to_float<<<grid_for(n, 256), 256, 0, s>>>(n, L.dinv, L.dinvf);
  return estimate_lmax<float>(L.A, L.dinvf, s, partials, sc.red, sc.h_red, stencil);
}

// named set-up phase for the per-kernel profile (no kernels of its own)
struct Phase {
  std::unique_ptr<ProfScope> p;
  cudaStream_t s;
  explicit Phase(cudaStream_t st) : s(st) {}
  void start(const char* name) {
    p.reset();
    p.reset(new ProfScope(name, 0.0, s, 0));
  }
  void stop() { p.reset(); }
};

void amg_build(Amg& amg, const Bsr& Ain, const double* Bin, int nns, const AmgParams& prm,
               cudaStream_t s) {
  Phase ph(s);
  ph.start("setup_copy");
  amg.release();
  amg.mixed = prm.mixed;
  amg.cheb_degree = prm.cheb_degree;
  amg.cheb_degree_coarse = prm.cheb_degree_coarse;
  amg.cheb_ratio = prm.cheb_ratio;
  amg.use_graph = prm.use_graph;
  SetupScratch sc;
  sc.err = dalloc<int>(4);
  PFF_CUDA(cudaMallocHost(&sc.h_err, sizeof(int) * 4));
  PFF_CUDA(cudaMallocHost(&sc.h_red, sizeof(double) * 4));
  sc.red = dalloc<double>(4);
  double* partials = dalloc<double>(RED_PARTIALS);
  PFF_CUDA(cudaMemsetAsync(sc.err, 0, sizeof(int) * 4, s));

  Bsr A;
  copy_bsr(Ain, A, s);
  int nb = A.nrows, br = A.br;
  double* B = dalloc<double>((size_t)nb * br * nns);
  PFF_CUDA(cudaMemcpyAsync(B, Bin, sizeof(double) * (size_t)nb * br * nns, cudaMemcpyDeviceToDevice, s));
  const int cd = prm.coord_dim;
  double* X = nullptr;   // node coordinates of the current level (distance strength)
  if (prm.coords && cd > 0) {
    X = dalloc<double>((size_t)nb * cd);
    PFF_CUDA(cudaMemcpyAsync(X, prm.coords, sizeof(double) * (size_t)nb * cd,
                             cudaMemcpyDeviceToDevice, s));
  }

  const AmgParams* fine_stencil = (prm.st || prm.stf) && prm.mesh.dim > 0 ? &prm : nullptr;
  for (int level = 0;; ++level) {
    const int n = nb * br;
    // a direct (dense) coarse solve only up to coarse_max rows; a larger level at the
    // level limit smooths only (below)
    if (n <= prm.coarse_max) {
      // coarsest level: dense inverse
      ph.start("setup_coarse_inverse");
      amg.nc = n;
      double* Dm = dalloc<double>((size_t)n * n);
      amg.cinv = dalloc<double>((size_t)n * n);
      PFF_CUDA(cudaMemsetAsync(Dm, 0, sizeof(double) * (size_t)n * n, s));
      count_launch();
      k_densify<<<grid_for(nb, 128), 128, 0, s>>>(nb, br, A.rowptr, A.col, A.val, Dm, n);
      count_launch(1 + 2 * n);
      k_gj_identity<<<grid_for((int64_t)n * n, 256), 256, 0, s>>>(n, amg.cinv);
      for (int k = 0; k < n; ++k) {
        k_gj_pivot<<<1, 256, 0, s>>>(n, k, Dm, amg.cinv, sc.err);
        k_gj_elim<<<n, 128, 0, s>>>(n, k, Dm, amg.cinv);
      }
      PFF_LAUNCH("coarse inverse");
      if (amg.mixed) {
        amg.cinvf = dalloc<float>((size_t)n * n);
        count_launch();
        k_to_float<<<grid_for((int64_t)n * n, 256), 256, 0, s>>>((int64_t)n * n, amg.cinv, amg.cinvf);
      }
      amg.cx = dalloc<double>(n);
      amg.cb = dalloc<double>(n);
      check_err(sc, s, "coarse inverse");
      dfree(Dm);
      A.release();
      break;
    }
    ph.start("setup_strength");
    AmgLevel L;
    L.A = A;   // takes ownership
    L.n = n;
    L.dinv = dalloc<double>(n);
    double* dnorm = dalloc<double>(nb);
    count_launch();
    k_diag<<<grid_for(nb, 256), 256, 0, s>>>(nb, br, A.rowptr, A.col, A.val, dnorm, L.dinv, sc.err);
    if (level >= prm.max_levels) {
      // level limit reached: this level only smooths (no strength or aggregation work)
      L.terminal = true;
      ph.start("setup_lmax");
      L.lmax = level_lmax(amg, L, s, partials, sc, level == 0 ? fine_stencil : nullptr);
      L.x = dalloc<double>(n);
      L.b = dalloc<double>(n);
      L.r = dalloc<double>(n);
      L.d = dalloc<double>(n);
      L.t = dalloc<double>(n);
      PFF_CUDA(cudaStreamSynchronize(s));
      dfree(dnorm);
      amg.lev.push_back(L);
      amg.nc = 0;
      break;
    }
    // strength
    uint8_t* s0 = dalloc<uint8_t>(A.nnzb);
    uint8_t* strong = dalloc<uint8_t>(A.nnzb);
    double* snorm = dalloc<double>(A.nnzb);
    if (X) {
      double* wmax = dalloc<double>(nb);
      count_launch(2);
      k_dist_wmax<<<grid_for(nb, 256), 256, 0, s>>>(nb, A.rowptr, A.col, X, cd, wmax);
      k_strength_dist<<<grid_for(nb, 256), 256, 0, s>>>(nb, br, A.rowptr, A.col, A.val, dnorm, X, cd,
                                                        wmax, prm.theta * prm.theta,
                                                        prm.mdrop * prm.mdrop, s0, snorm);
      PFF_CUDA(cudaStreamSynchronize(s));
      dfree(wmax);
    } else {
      count_launch();
      k_strength<<<grid_for(nb, 256), 256, 0, s>>>(nb, br, A.rowptr, A.col, A.val, dnorm,
                                                   prm.theta * prm.theta, s0, snorm);
    }
    count_launch();
    k_symmetrize<<<grid_for(nb, 256), 256, 0, s>>>(nb, A.rowptr, A.col, s0, strong);
    PFF_LAUNCH("strength");
    // MIS(2)
    ph.start("setup_mis2");
    int* state = dalloc<int>(nb);
    uint8_t* iso = dalloc<uint8_t>(nb);
    unsigned long long* M1 = dalloc<unsigned long long>(nb);
    unsigned long long* M2 = dalloc<unsigned long long>(nb);
    int* und = dalloc<int>(1);
    int* h_und = sc.h_err + 1;
    count_launch();
    k_mis_init<<<grid_for(nb, 256), 256, 0, s>>>(nb, A.rowptr, strong, state, iso);
    int rounds = 0;
    for (;; ++rounds) {
      PFF_CUDA(cudaMemsetAsync(und, 0, sizeof(int), s));
      count_launch();
      k_mis_max1<<<grid_for(nb, 256), 256, 0, s>>>(nb, A.rowptr, A.col, strong, state, M1);
      count_launch();
      k_mis_max2<<<grid_for(nb, 256), 256, 0, s>>>(nb, A.rowptr, A.col, strong, M1, M2);
      count_launch();
      k_mis_decide<<<grid_for(nb, 256), 256, 0, s>>>(nb, state, M2, und);
      PFF_LAUNCH("mis");
      PFF_CUDA(cudaMemcpyAsync(h_und, und, sizeof(int), cudaMemcpyDeviceToHost, s));
      PFF_CUDA(cudaStreamSynchronize(s));
      if (*h_und == 0) break;
      if (rounds > 200) fail(PFF_ERR_CAPACITY, "AMG MIS(2) did not terminate");
    }
    // aggregates
    ph.start("setup_aggregate");
    int* flag = dalloc<int>(nb + 1);
    int* rootid = dalloc<int>(nb + 1);
    count_launch();
    k_root_flags<<<grid_for(nb, 256), 256, 0, s>>>(nb, state, flag);
    int nagg = 0;
    exclusive_scan_int(flag, rootid, nb, &nagg, s);
    int* agg1 = dalloc<int>(nb);
    int* agg = dalloc<int>(nb);
    count_launch();
    k_agg_pass1<<<grid_for(nb, 256), 256, 0, s>>>(nb, A.rowptr, A.col, strong, snorm, state, iso,
                                                  rootid, agg1);
    count_launch();
    k_agg_pass2<<<grid_for(nb, 256), 256, 0, s>>>(nb, A.rowptr, A.col, strong, snorm, agg1, agg);
    PFF_LAUNCH("aggregate");
    if (nagg == 0 || (int64_t)nagg * nns > (int64_t)(0.9 * n) || level >= prm.max_levels) {
      // every row is isolated (identity / decoupled rows): smoothing is all there is
      L.terminal = true;
      L.lmax = level_lmax(amg, L, s, partials, sc, level == 0 ? fine_stencil : nullptr);
      L.x = dalloc<double>(n);
      L.b = dalloc<double>(n);
      L.r = dalloc<double>(n);
      L.d = dalloc<double>(n);
      L.t = dalloc<double>(n);
      PFF_CUDA(cudaStreamSynchronize(s));
      dfree(dnorm);
      dfree(s0);
      dfree(strong);
      dfree(snorm);
      dfree(state);
      dfree(iso);
      dfree(M1);
      dfree(M2);
      dfree(und);
      dfree(flag);
      dfree(rootid);
      dfree(agg1);
      dfree(agg);
      amg.lev.push_back(L);
      amg.nc = 0;
      break;
    }
    int* cnt = dalloc<int>(nagg + 1);
    int* off = dalloc<int>(nagg + 1);
    int* cursor = dalloc<int>(nagg + 1);
    int* members = dalloc<int>(nb);
    PFF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (nagg + 1), s));
    PFF_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int) * (nagg + 1), s));
    count_launch();
    k_count_members<<<grid_for(nb, 256), 256, 0, s>>>(nb, agg, cnt);
    int nmem = 0;
    exclusive_scan_int(cnt, off, nagg, &nmem, s);
    count_launch();
    k_fill_members<<<grid_for(nb, 256), 256, 0, s>>>(nb, agg, off, cursor, members);
    count_launch();
    k_sort_segments<<<grid_for(nagg, 128), 128, 0, s>>>(nagg, off, members, nullptr);
    // tentative prolongator + coarse near-null space
    ph.start("setup_tentative");
    double* Qn = dalloc<double>((size_t)nb * br * nns);
    double* Bc = dalloc<double>((size_t)nagg * nns * nns);
    count_launch();
    k_zero_rows<<<grid_for(nb, 256), 256, 0, s>>>(nb, br * nns, agg, Qn);
    count_launch();
    k_tentative<<<grid_for(nagg, 64), 64, 0, s>>>(nagg, br, nns, off, members, B, (int64_t)nb * br,
                                                  Qn, Bc, (int64_t)nagg * nns);
    PFF_LAUNCH("tentative");
    double* Xc = nullptr;
    if (X) {
      Xc = dalloc<double>((size_t)nagg * cd);
      count_launch();
      k_centroids<<<grid_for(nagg, 128), 128, 0, s>>>(nagg, off, members, X, cd, Xc);
      PFF_LAUNCH("centroids");
    }
    // smoothed prolongator
    ph.start("setup_lmax");
    L.lmax = level_lmax(amg, L, s, partials, sc, level == 0 ? fine_stencil : nullptr);
    ph.start("setup_prolongator");
    const double omega = 4.0 / (3.0 * L.lmax);
    Bsr& P = L.P;
    P.nrows = nb;
    P.ncols = nagg;
    P.br = br;
    P.bc = nns;
    P.rowptr = dalloc<int>(nb + 1);
    int* pc = dalloc<int>(nb + 1);
    count_launch();
    k_P_count<<<grid_for(nb, 128), 128, 0, s>>>(nb, A.rowptr, A.col, strong, agg, pc, sc.err);
    int pnnz = 0;
    exclusive_scan_int(pc, P.rowptr, nb, &pnnz, s);
    P.nnzb = pnnz;
    P.col = dalloc<int>(pnnz);
    P.val = dalloc<double>((size_t)pnnz * br * nns);
    count_launch();
    k_P_fill<<<grid_for(nb, 128), 128, 0, s>>>(nb, br, nns, A.rowptr, A.col, A.val, strong, agg, Qn,
                                               L.dinv, omega, P.rowptr, P.col, P.val);
    PFF_LAUNCH("P");
    check_err(sc, s, "prolongator");
    transpose(P, L.R, s);
    // Galerkin product
    ph.start("setup_galerkin");
    Bsr AP, Ac;
    spgemm(L.A, P, AP, sc.err, s);
    spgemm(L.R, AP, Ac, sc.err, s);
    check_err(sc, s, "Galerkin product");
    count_launch();
    k_fix_diag<<<grid_for(Ac.nrows, 128), 128, 0, s>>>(Ac.nrows, Ac.br, Ac.rowptr, Ac.col, Ac.val);
    PFF_LAUNCH("fix_diag");
    AP.release();
    // work vectors and FP32 copies
    ph.start("setup_vectors");
    L.x = dalloc<double>(n);
    L.b = dalloc<double>(n);
    L.r = dalloc<double>(n);
    L.d = dalloc<double>(n);
    L.t = dalloc<double>(n);
    if (amg.mixed) {   // (A and dinv were copied to FP32 for the eigenvalue estimate)
      make_float(L.P, s);
      make_float(L.R, s);
    }
    PFF_CUDA(cudaStreamSynchronize(s));
    dfree(dnorm);
    dfree(s0);
    dfree(strong);
    dfree(snorm);
    dfree(state);
    dfree(iso);
    dfree(M1);
    dfree(M2);
    dfree(und);
    dfree(flag);
    dfree(rootid);
    dfree(agg1);
    dfree(agg);
    dfree(cnt);
    dfree(off);
    dfree(cursor);
    dfree(members);
    dfree(Qn);
    dfree(pc);
    dfree(B);
    dfree(X);
    amg.lev.push_back(L);
    // next level
    A = Ac;
    B = Bc;
    X = Xc;
    nb = Ac.nrows;
    br = Ac.br;
  }
  dfree(B);
  dfree(X);
  dfree(partials);
  dfree(sc.err);
  dfree(sc.red);
  cudaFreeHost(sc.h_err);
  cudaFreeHost(sc.h_red);
  ph.start("setup_autotune");
  for (auto& L : amg.lev) {
    L.A.group = L.P.group = L.R.group = prm.spmv_group;
    if (prm.spmv_group == BSR_SELL && amg.mixed) {
      bsr_make_sell(L.A, s);
      bsr_make_sell(L.P, s);
      bsr_make_sell(L.R, s);
    }
    if (prm.spmv_group == 0) {
      // the finest operator is applied through its stencil when L.stencil is set;
      // its BSR copy is timed all the same (it is cheap and rarely used)
      bsr_autotune(L.A, amg.mixed, s);
      bsr_autotune(L.P, amg.mixed, s);
      bsr_autotune(L.R, amg.mixed, s);
    }
  }
  ph.stop();
  amg.built = 1;
  static std::atomic<uint64_t> builds{0};
  amg.build_id = ++builds;
  if (verbose()) {
    std::fprintf(stderr, "[pff] AMG (%s): %zu levels + coarse %d\n", amg.mixed ? "fp32" : "fp64",
                 amg.lev.size(), amg.nc);
    for (size_t l = 0; l < amg.lev.size(); ++l) {
      const auto& L = amg.lev[l];
      std::fprintf(stderr, "[pff]   level %zu: rows %d (block %d) nnzb %lld lmax %.4g%s\n", l,
                   L.A.nrows, L.A.br, (long long)L.A.nnzb, L.lmax, L.terminal ? " terminal" : "");
    }
  }
}

void amg_vcycle(Amg& amg, const double* r, double* z, cudaStream_t s) {
  if (amg.lev.empty()) {
    // whole problem is the coarse level
    ProfScope ps("coarse_solve", 8.0 * amg.nc * (amg.nc + 2.0), s);
    k_dense_mv<double><<<grid_for(amg.nc, 8), 256, 0, s>>>(amg.nc, amg.cinv, r, z);
    PFF_LAUNCH("coarse only");
    return;
  }
  AmgLevel& L0 = amg.lev[0];
  const int64_t n = L0.n;
  if (amg.mixed && L0.stencil) {
    // the first and last level-0 smoothing steps convert r and z themselves
    vcycle_level<float>(amg, 0, reinterpret_cast<float*>(L0.b), reinterpret_cast<float*>(L0.x), s,
                        r, z);
  } else if (amg.mixed) {
    float* b = reinterpret_cast<float*>(L0.b);
    float* x = reinterpret_cast<float*>(L0.x);
    {
      ProfScope ps("convert", 12.0 * n, s);
      k_convert<double, float><<<grid_for(n, 256), 256, 0, s>>>(n, r, b);
    }
    vcycle_level<float>(amg, 0, b, x, s);
    ProfScope ps("convert", 12.0 * n, s);
    k_convert<float, double><<<grid_for(n, 256), 256, 0, s>>>(n, x, z);
  } else {
    PFF_CUDA(cudaMemcpyAsync(L0.b, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    vcycle_level<double>(amg, 0, L0.b, L0.x, s);
    PFF_CUDA(cudaMemcpyAsync(z, L0.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  PFF_LAUNCH("vcycle");
}

}  // namespace pff
