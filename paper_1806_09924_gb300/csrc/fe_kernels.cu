// Element-batched Q1 kernels for Formulation 1 (Section 2) and the Jacobian
// blocks of Section 3.1 on tensor-product meshes.
//
// Every output is owned by one thread: a node's rows are gathered by that node's
// thread from its 2^d adjacent cells, so results are written once, without
// atomics, and are bitwise reproducible.  The residual and the phase-field
// assembly first evaluate each cell's Gauss points once (one thread per cell,
// records in global memory) and then gather; the other kernels recompute the
// cell quantities they need per node.  Cells are axis-aligned boxes, so the
// reference-to-physical map is diagonal (d/dx_l = (1/h_l) d/dxi_l); the
// quadrature is the tensor 2^d-point Gauss rule.  Quadrature-point values use
// the interpolated nodal phi, phi~ (then squared).
//
// Stencil layout: the Jacobian rows of node i couple to the 3^d neighbours
// (i_x + o_x, i_y + o_y[, i_z + o_z]), o in {-1,0,1}; slot s = (o_x+1) +
// 3(o_y+1) + 9(o_z+1) (increasing neighbour index).  Values are stored slot-
// major so that consecutive threads read consecutive addresses:
//   Kuu[((s*d + m)*d + n)*N + i]   (M_uu, d x d block per slot)
//   Kpu[(s*d + n)*N + i]           (M_phi_u)
//   Kpp[s*N + i]                   (M_phi_phi)
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "pff_internal.h"

namespace pff {

namespace {

constexpr int BLK = 128;

__device__ __forceinline__ double gauss_pt(int i) {
  return i ? 0.78867513459481288225 : 0.21132486540518711775;   // (1 +- 1/sqrt 3) / 2
}

// Q1 shape value of local node a at Gauss point q of [0,1]^D
template <int D>
__device__ __forceinline__ double shp(int a, int q) {
  double r = 1.0;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const double x = gauss_pt((q >> l) & 1);
    r *= ((a >> l) & 1) ? x : 1.0 - x;
  }
  return r;
}

// reference derivative d N_a / d xi_l at Gauss point q
template <int D>
__device__ __forceinline__ double dshp(int a, int q, int l) {
  double r = ((a >> l) & 1) ? 1.0 : -1.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k == l) continue;
    const double x = gauss_pt((q >> k) & 1);
    r *= ((a >> k) & 1) ? x : 1.0 - x;
  }
  return r;
}

template <int D>
__device__ __forceinline__ void node_index(int64_t i, const MeshDev& m, int* idx) {
  idx[0] = (int)(i % m.nn[0]);
  const int64_t r = i / m.nn[0];
  if (D == 2) {
    idx[1] = (int)r;
  } else {
    idx[1] = (int)(r % m.nn[1]);
    idx[2] = (int)(r / m.nn[1]);
  }
}

template <int D>
__device__ __forceinline__ bool is_boundary(const int* idx, const MeshDev& m) {
  bool b = false;
#pragma unroll
  for (int l = 0; l < D; ++l) b |= (idx[l] == 0) | (idx[l] == m.nn[l] - 1);
  return b;
}

template <int D>
__device__ __forceinline__ int64_t node_of(const int* idx, const MeshDev& m) {
  int64_t r = idx[0] + (int64_t)m.nn[0] * idx[1];
  if (D == 3) r += (int64_t)m.nn[0] * m.nn[1] * idx[2];
  return r;
}

// Cell c adjacent to node idx: offset bit l of c = cell index - node index + 1.
// Returns false if the cell lies outside the mesh.  ci receives the cell index,
// h the edge lengths, and the node's local index inside the cell is (~c) & (2^D-1).
template <int D>
__device__ __forceinline__ bool adjacent_cell(const int* idx, int c, const MeshDev& m, int* ci,
                                              double* h) {
#pragma unroll
  for (int l = 0; l < D; ++l) {
    ci[l] = idx[l] - 1 + ((c >> l) & 1);
    if (ci[l] < 0 || ci[l] >= m.nc[l]) return false;
  }
#pragma unroll
  for (int l = 0; l < D; ++l) h[l] = m.X[l][ci[l] + 1] - m.X[l][ci[l]];
  return true;
}

template <int D>
__device__ __forceinline__ int64_t cell_node(const int* ci, int b, const MeshDev& m) {
  int64_t r = ci[0] + (b & 1) + (int64_t)m.nn[0] * (ci[1] + ((b >> 1) & 1));
  if (D == 3) r += (int64_t)m.nn[0] * m.nn[1] * (ci[2] + ((b >> 2) & 1));
  return r;
}

template <int D>
__device__ __forceinline__ bool node_on_boundary(const int* ci, int b, const MeshDev& m) {
  bool r = false;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const int k = ci[l] + ((b >> l) & 1);
    r |= (k == 0) | (k == m.nn[l] - 1);
  }
  return r;
}

// stencil slot of trial node b of a cell at offset c relative to the row node
template <int D>
__device__ __forceinline__ int slot_of(int c, int b) {
  int s = 0, mul = 1;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const int o = ((c >> l) & 1) + ((b >> l) & 1);   // offset + 1 in {0,1,2}
    s += o * mul;
    mul *= 3;
  }
  return s;
}

// ------------------------------------------------------------- residual ---
// F = -r(U), r = left-hand sides of Eq. (E22ATW) / (E33ATW) tested with chi_i.
//
// Two passes.  k_residual_qp evaluates, once per cell and Gauss point q, every
// quantity the test functions are integrated against, already scaled by the
// quadrature weight and the inverse edge lengths:
//   T[a][l] = JxW (g(phi~) sigma(u)[a][l] + phi^2 p delta_al) / h_l   (stress + pressure)
//   s0      = JxW ((1-kappa) phi sigma:e + 2 phi p div u - G_c/eps (1-phi))
//   gg[l]   = JxW G_c eps (d phi / dx_l) / h_l
// so that node a of the cell receives  r_u[a'] += sum_l T[a'][l] dN_a/dxi_l  and
// r_phi += s0 N_a + sum_l gg[l] dN_a/dxi_l  (reference-cell derivatives).
// k_residual_gather then sums, for each node, its 2^d cells' records in a fixed
// order.  Records are stored slot-major (QP[(q R + r) n_cells + cell]) so both
// passes read and write coalesced.
template <int D>
__host__ __device__ constexpr int res_rec() { return D * D + D + 1; }

template <int D>
__device__ __forceinline__ void cell_index(int64_t cl, const MeshDev& m, int* ci) {
  ci[0] = (int)(cl % m.nc[0]);
  const int64_t r = cl / m.nc[0];
  if (D == 2) {
    ci[1] = (int)r;
  } else {
    ci[1] = (int)(r % m.nc[1]);
    ci[2] = (int)(r / m.nc[1]);
  }
}

template <int D>
__device__ __forceinline__ int64_t cell_of(const int* ci, const MeshDev& m) {
  int64_t r = ci[0] + (int64_t)m.nc[0] * ci[1];
  if (D == 3) r += (int64_t)m.nc[0] * m.nc[1] * ci[2];
  return r;
}

// Cell adjacent to node idx at offset c (bit l = cell index - node index + 1);
// false outside the mesh.
template <int D>
__device__ __forceinline__ bool adjacent_cell_index(const int* idx, int c, const MeshDev& m,
                                                    int* ci) {
  bool in = true;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    ci[l] = idx[l] - 1 + ((c >> l) & 1);
    in &= (ci[l] >= 0) & (ci[l] < m.nc[l]);
  }
  return in;
}

template <int D, int TB = BLK>
__global__ void __launch_bounds__(TB) k_residual_qp(MeshDev m, Material mat, int64_t ncell,
                                                     const double* __restrict__ u,
                                                     const double* __restrict__ phi,
                                                     const double* __restrict__ phit,
                                                     double* __restrict__ QP) {
  const int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cl >= ncell) return;
  constexpr int NA = 1 << D, R = res_rec<D>();
  const double wq = D == 2 ? 0.25 : 0.125;
  int ci[3];
  cell_index<D>(cl, m, ci);
  double ih[D], vol = 1.0;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const double h = m.X[l][ci[l] + 1] - m.X[l][ci[l]];
    ih[l] = 1.0 / h;
    vol *= h;
  }
  double ue[NA][D], pe[NA], te[NA];
#pragma unroll
  for (int b = 0; b < NA; ++b) {
    const int64_t nb = cell_node<D>(ci, b, m);
#pragma unroll
    for (int a = 0; a < D; ++a) ue[b][a] = u[nb * D + a];
    pe[b] = phi[nb];
    te[b] = phit[nb];
  }
  const double JxW = wq * vol;
  const double k1 = 1.0 - mat.kappa;
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    double G[D][D], gp[D], ph = 0.0, pt = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      gp[a] = 0.0;
#pragma unroll
      for (int l = 0; l < D; ++l) G[a][l] = 0.0;
    }
#pragma unroll
    for (int b = 0; b < NA; ++b) {
      const double Nb = shp<D>(b, q);
      ph += Nb * pe[b];
      pt += Nb * te[b];
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const double dN = dshp<D>(b, q, l);   // reference derivative; 1/h_l applied below
        gp[l] += dN * pe[b];
#pragma unroll
        for (int a = 0; a < D; ++a) G[a][l] += ue[b][a] * dN;
      }
    }
#pragma unroll
    for (int l = 0; l < D; ++l) {
      gp[l] *= ih[l];
#pragma unroll
      for (int a = 0; a < D; ++a) G[a][l] *= ih[l];
    }
    double div = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) div += G[l][l];
    double sig[D][D], sige = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const double e = 0.5 * (G[a][l] + G[l][a]);
        sig[a][l] = 2.0 * mat.mu * e + (a == l ? mat.lam * div : 0.0);
        sige += sig[a][l] * e;
      }
    const double g = k1 * pt * pt + mat.kappa;
    const double pp = ph * ph * mat.p;
    double* out = QP + (int64_t)q * R * ncell + cl;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int l = 0; l < D; ++l)
        out[(a * D + l) * ncell] = JxW * (g * sig[a][l] + (a == l ? pp : 0.0)) * ih[l];
    out[D * D * ncell] =
        JxW * (k1 * ph * sige + 2.0 * ph * mat.p * div - mat.Gc / mat.eps * (1.0 - ph));
#pragma unroll
    for (int l = 0; l < D; ++l) out[(D * D + 1 + l) * ncell] = JxW * mat.Gc * mat.eps * gp[l] * ih[l];
  }
}

template <int D, int TB = BLK>
__global__ void __launch_bounds__(TB) k_residual_gather(MeshDev m, int64_t n, int64_t ncell,
                                                         const double* __restrict__ QP,
                                                         double* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NA = 1 << D, R = res_rec<D>();
  int idx[3];
  node_index<D>(i, m, idx);
  double ru[D], rp = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) ru[a] = 0.0;
#pragma unroll
  for (int c = 0; c < NA; ++c) {
    int ci[3];
    if (!adjacent_cell_index<D>(idx, c, m, ci)) continue;
    const int ai = (~c) & (NA - 1);
    const double* rec = QP + cell_of<D>(ci, m);
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const double* r = rec + (int64_t)q * R * ncell;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int l = 0; l < D; ++l) ru[a] += __ldg(r + (a * D + l) * ncell) * dshp<D>(ai, q, l);
      rp += __ldg(r + D * D * ncell) * shp<D>(ai, q);
#pragma unroll
      for (int l = 0; l < D; ++l) rp += __ldg(r + (D * D + 1 + l) * ncell) * dshp<D>(ai, q, l);
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) F[i * D + a] = -ru[a];
  F[(int64_t)D * n + i] = -rp;
}

// ---------------------------------------------------------- phi~, mass, S ---
__global__ void k_phi_tilde(int64_t n, int first, const double* __restrict__ phi_old,
                            const double* __restrict__ phi_prev, double* __restrict__ phit) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (first) {
    phit[i] = phi_old[i];
  } else {
    const double v = 2.0 * phi_old[i] - phi_prev[i];
    phit[i] = fmin(fmax(v, 0.0), 1.0);
  }
}

// mass[i] = (1, chi_i); optionally S_phi[i] = G_c (chi_i, chi_i)/eps + G_c eps |grad chi_i|^2
template <int D>
__global__ void k_mass_and_sphi(MeshDev m, Material mat, int64_t n, double* __restrict__ mass,
                                double* __restrict__ Sphi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NA = 1 << D;
  const double wq = D == 2 ? 0.25 : 0.125;
  int idx[3];
  node_index<D>(i, m, idx);
  double ms = 0.0, mm = 0.0, kk = 0.0;
  for (int c = 0; c < NA; ++c) {
    int ci[3];
    double h[3];
    if (!adjacent_cell<D>(idx, c, m, ci, h)) continue;
    const int ai = (~c) & (NA - 1);
    double vol = 1.0;
    for (int l = 0; l < D; ++l) vol *= h[l];
    const double JxW = wq * vol;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const double Na = shp<D>(ai, q);
      ms += JxW * Na;
      mm += JxW * Na * Na;
      double g2 = 0.0;
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const double d = dshp<D>(ai, q, l) / h[l];
        g2 += d * d;
      }
      kk += JxW * g2;
    }
  }
  if (mass) mass[i] = ms;
  if (Sphi) Sphi[i] = mat.Gc * (mm / mat.eps + mat.eps * kk);
}

template <int D>
__global__ void k_scaling_u(int64_t n, const double* __restrict__ Kuu, double* __restrict__ S,
                            double* __restrict__ Sinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int center = D == 2 ? 4 : 13;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const double v = Kuu[((int64_t)(center * D + a) * D + a) * n + i];
    S[i * D + a] = v;
    Sinv[i * D + a] = 1.0 / v;
  }
}

__global__ void k_invert(int64_t n, const double* __restrict__ S, double* __restrict__ Sinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Sinv[i] = 1.0 / S[i];
}

// --------------------------------------------------------------- assembly ---
// (M_uu)_ij = (g(phi~) sigma(chi_j), e(chi_i)); Dirichlet rows -> identity,
// Dirichlet columns -> 0.
template <int D, int TB = BLK>
__global__ void __launch_bounds__(TB) k_assemble_uu(MeshDev m, Material mat, int64_t n,
                                                     const double* __restrict__ phit,
                                                     double* __restrict__ Kuu) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NA = 1 << D;
  constexpr int NS = D == 2 ? 9 : 27;
  constexpr int center = D == 2 ? 4 : 13;
  const double wq = D == 2 ? 0.25 : 0.125;
  int idx[3];
  node_index<D>(i, m, idx);
  for (int s = 0; s < NS * D * D; ++s) Kuu[(int64_t)s * n + i] = 0.0;
  if (is_boundary<D>(idx, m)) {
    for (int a = 0; a < D; ++a) Kuu[((int64_t)(center * D + a) * D + a) * n + i] = 1.0;
    return;
  }
  const double k1 = 1.0 - mat.kappa;
#pragma unroll 1
  for (int c = 0; c < NA; ++c) {
    int ci[3];
    double h[3];
    if (!adjacent_cell<D>(idx, c, m, ci, h)) continue;
    const int ai = (~c) & (NA - 1);
    double ih[D], vol = 1.0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
      ih[l] = 1.0 / h[l];
      vol *= h[l];
    }
    double te[NA];
#pragma unroll
    for (int b = 0; b < NA; ++b) te[b] = phit[cell_node<D>(ci, b, m)];
    const double JxW = wq * vol;
    // per Gauss point: the degraded weight and the test node's gradient
    double wg[NA], dNa[NA][D];
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      double pt = 0.0;
#pragma unroll
      for (int b = 0; b < NA; ++b) pt += shp<D>(b, q) * te[b];
      wg[q] = JxW * (k1 * pt * pt + mat.kappa);
#pragma unroll
      for (int l = 0; l < D; ++l) dNa[q][l] = dshp<D>(ai, q, l) * ih[l];
    }
    // one trial node's D x D block at a time, summed over the Gauss points in order
    // (only D x D accumulators live: no spills in 3d)
#pragma unroll 1
    for (int b = 0; b < NA; ++b) {
      if (node_on_boundary<D>(ci, b, m)) continue;
      double Kb[D][D];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int e = 0; e < D; ++e) Kb[a][e] = 0.0;
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        double dNb[D], dd = 0.0;
#pragma unroll
        for (int l = 0; l < D; ++l) {
          dNb[l] = dshp<D>(b, q, l) * ih[l];
          dd += dNa[q][l] * dNb[l];
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int e = 0; e < D; ++e)
            Kb[a][e] += wg[q] * (mat.mu * ((a == e ? dd : 0.0) + dNa[q][e] * dNb[a]) +
                                 mat.lam * dNa[q][a] * dNb[e]);
      }
      const int s = slot_of<D>(c, b);
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int e = 0; e < D; ++e) Kuu[((int64_t)(s * D + a) * D + e) * n + i] += Kb[a][e];
    }
  }
}

// (M_phi_u)_ij = 2(1-kappa)(phi sigma(chi_j^u):e(u), chi_i) + 2p(phi div chi_j^u, chi_i)
// (M_phi_phi)_ij = ((1-kappa) sigma(u):e(u) + 2p div u + G_c/eps) (chi_j, chi_i)
//                 + G_c eps (grad chi_j, grad chi_i)
// Dirichlet displacement columns of M_phi_u are zero (eliminated DoFs).
//
// Two passes, as for the residual.  k_assemble_phi_qp stores per cell and Gauss
// point q
//   M[e][l] = JxW (2(1-kappa) phi sigma(u)[e][l] + 2 p phi delta_el) / h_l
//   w0      = JxW ((1-kappa) sigma:e + 2 p div u + G_c/eps)
// and k_assemble_phi_gather forms the rows of node a from its 2^d cells:
//   M_phi_u[a][(b,e)] += sum_q N_a sum_l M[e][l] dN_b/dxi_l,
//   M_phi_phi[a][b]   += sum_q w0 N_a N_b
//                        + G_c eps JxW sum_q sum_l dN_a/dxi_l dN_b/dxi_l / h_l^2
// (the last term depends on the cell's edge lengths only and is formed in the
// gather).  The sums over q for all trial nodes b at once use the tensor-product
// structure of the Q1 basis (sum factorisation, below).
template <int D>
__host__ __device__ constexpr int phi_rec() { return D * D + 1; }

// out[b] = sum_q A[q] N_b(q) for every local node b: the 2^D x 2^D shape-value
// matrix is a Kronecker product of D 2 x 2 factors s(b_k, q_k) (s(0,q) = 1 - x_q,
// s(1,q) = x_q), applied one axis at a time.
template <int D>
__device__ __forceinline__ void contract_shp(double (&W)[1 << D]) {
  constexpr int NA = 1 << D;
  const double x0 = gauss_pt(0), x1 = gauss_pt(1);
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      if ((q >> k) & 1) continue;
      const double v0 = W[q], v1 = W[q | (1 << k)];
      W[q] = (1.0 - x0) * v0 + (1.0 - x1) * v1;
      W[q | (1 << k)] = x0 * v0 + x1 * v1;
    }
}

// out[b] += sum_q A[q] dN_b/dxi_l(q) for every b.  dN_b/dxi_l = sign(b_l) times
// the product over the other axes of s(b_k, q_k), which does not depend on q_l:
// sum A over q_l first, apply the other axes' factors, then the sign.
template <int D>
__device__ __forceinline__ void contract_dshp_add(int l, const double (&A)[1 << D],
                                                  double (&out)[1 << D]) {
  constexpr int NA = 1 << D;
  const double x0 = gauss_pt(0), x1 = gauss_pt(1);
  double W[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) W[q] = ((q >> l) & 1) ? 0.0 : A[q] + A[q | (1 << l)];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (k == l) continue;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      if (((q >> k) & 1) || ((q >> l) & 1)) continue;
      const double v0 = W[q], v1 = W[q | (1 << k)];
      W[q] = (1.0 - x0) * v0 + (1.0 - x1) * v1;
      W[q | (1 << k)] = x0 * v0 + x1 * v1;
    }
  }
#pragma unroll
  for (int b = 0; b < NA; ++b) {
    const double v = W[b & ~(1 << l)];
    out[b] += ((b >> l) & 1) ? v : -v;
  }
}

template <int D, int TB = BLK>
__global__ void __launch_bounds__(TB) k_assemble_phi_qp(MeshDev m, Material mat, int64_t ncell,
                                                         const double* __restrict__ u,
                                                         const double* __restrict__ phi,
                                                         double* __restrict__ QP) {
  const int64_t cl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cl >= ncell) return;
  constexpr int NA = 1 << D, R = phi_rec<D>();
  const double wq = D == 2 ? 0.25 : 0.125;
  int ci[3];
  cell_index<D>(cl, m, ci);
  double ih[D], vol = 1.0;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    const double h = m.X[l][ci[l] + 1] - m.X[l][ci[l]];
    ih[l] = 1.0 / h;
    vol *= h;
  }
  double ue[NA][D], pe[NA];
#pragma unroll
  for (int b = 0; b < NA; ++b) {
    const int64_t nb = cell_node<D>(ci, b, m);
#pragma unroll
    for (int a = 0; a < D; ++a) ue[b][a] = u[nb * D + a];
    pe[b] = phi[nb];
  }
  const double JxW = wq * vol;
  const double k1 = 1.0 - mat.kappa;
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    double G[D][D], ph = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int l = 0; l < D; ++l) G[a][l] = 0.0;
#pragma unroll
    for (int b = 0; b < NA; ++b) {
      ph += shp<D>(b, q) * pe[b];
#pragma unroll
      for (int l = 0; l < D; ++l)
#pragma unroll
        for (int a = 0; a < D; ++a) G[a][l] += ue[b][a] * dshp<D>(b, q, l);
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int l = 0; l < D; ++l) G[a][l] *= ih[l];
    double div = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) div += G[l][l];
    double sig[D][D], sige = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const double e = 0.5 * (G[a][l] + G[l][a]);
        sig[a][l] = 2.0 * mat.mu * e + (a == l ? mat.lam * div : 0.0);
        sige += sig[a][l] * e;
      }
    const double cs = 2.0 * k1 * ph, cp = 2.0 * mat.p * ph;
    double* out = QP + (int64_t)q * R * ncell + cl;
#pragma unroll
    for (int e = 0; e < D; ++e)
#pragma unroll
      for (int l = 0; l < D; ++l)
        out[(e * D + l) * ncell] = JxW * (cs * sig[e][l] + (e == l ? cp : 0.0)) * ih[l];
    out[D * D * ncell] = JxW * (k1 * sige + 2.0 * mat.p * div + mat.Gc / mat.eps);
  }
}

template <int D, int TB = BLK>
__global__ void __launch_bounds__(TB) k_assemble_phi_gather(MeshDev m, Material mat, int64_t n,
                                                             int64_t ncell,
                                                             const double* __restrict__ QP,
                                                             double* __restrict__ Kpu,
                                                             double* __restrict__ Kpp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NA = 1 << D, R = phi_rec<D>();
  constexpr int NS = D == 2 ? 9 : 27;
  const double wq = D == 2 ? 0.25 : 0.125;
  int idx[3];
  node_index<D>(i, m, idx);
  for (int s = 0; s < NS * D; ++s) Kpu[(int64_t)s * n + i] = 0.0;
  for (int s = 0; s < NS; ++s) Kpp[(int64_t)s * n + i] = 0.0;
#pragma unroll 1
  for (int c = 0; c < NA; ++c) {
    int ci[3];
    if (!adjacent_cell_index<D>(idx, c, m, ci)) continue;
    const int ai = (~c) & (NA - 1);
    double kl[D], vol = 1.0;
#pragma unroll
    for (int l = 0; l < D; ++l) {
      const double h = m.X[l][ci[l] + 1] - m.X[l][ci[l]];
      kl[l] = 1.0 / (h * h);
      vol *= h;
    }
    const double gl = mat.Gc * mat.eps * wq * vol;
    const double* rec = QP + cell_of<D>(ci, m);
    double Na[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) Na[q] = shp<D>(ai, q);
    double Kpu_e[D][NA], Kpp_e[NA], A[NA];
#pragma unroll
    for (int b = 0; b < NA; ++b) {
#pragma unroll
      for (int e = 0; e < D; ++e) Kpu_e[e][b] = 0.0;
    }
#pragma unroll
    for (int e = 0; e < D; ++e)
#pragma unroll
      for (int l = 0; l < D; ++l) {
#pragma unroll
        for (int q = 0; q < NA; ++q)
          A[q] = Na[q] * __ldg(rec + ((int64_t)q * R + e * D + l) * ncell);
        contract_dshp_add<D>(l, A, Kpu_e[e]);
      }
    // mass-like part: sum_q w0 N_a N_b
#pragma unroll
    for (int q = 0; q < NA; ++q) Kpp_e[q] = Na[q] * __ldg(rec + ((int64_t)q * R + D * D) * ncell);
    contract_shp<D>(Kpp_e);
    // Laplace part: G_c eps JxW / h_l^2 sum_q dN_a/dxi_l dN_b/dxi_l
#pragma unroll
    for (int l = 0; l < D; ++l) {
      const double w = gl * kl[l];
#pragma unroll
      for (int q = 0; q < NA; ++q) A[q] = w * dshp<D>(ai, q, l);
      contract_dshp_add<D>(l, A, Kpp_e);
    }
#pragma unroll
    for (int b = 0; b < NA; ++b) {
      const int s = slot_of<D>(c, b);
      Kpp[(int64_t)s * n + i] += Kpp_e[b];
      if (node_on_boundary<D>(ci, b, m)) continue;
#pragma unroll
      for (int e = 0; e < D; ++e) Kpu[(int64_t)(s * D + e) * n + i] += Kpu_e[e][b];
    }
  }
}

// neighbour node of slot s, or -1 outside the mesh
template <int D>
__device__ __forceinline__ int64_t neighbour(const int* idx, int s, const MeshDev& m) {
  int o[3];
  o[0] = s % 3 - 1;
  o[1] = (s / 3) % 3 - 1;
  o[2] = s / 9 - 1;
  int j[3];
#pragma unroll
  for (int l = 0; l < D; ++l) {
    j[l] = idx[l] + o[l];
    if (j[l] < 0 || j[l] >= m.nn[l]) return -1;
  }
  return node_of<D>(j, m);
}

// Reduced right-hand side and active-set masking of the phase-field rows.
template <int D>
__global__ void k_reduce_phi(MeshDev m, int64_t n, const uint8_t* __restrict__ active,
                             const double* __restrict__ phi, const double* __restrict__ phi_old,
                             const double* __restrict__ F, double* __restrict__ Ft,
                             double* __restrict__ dUA, double* __restrict__ Kpu,
                             double* __restrict__ Kpp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NS = D == 2 ? 9 : 27;
  constexpr int center = D == 2 ? 4 : 13;
  int idx[3];
  node_index<D>(i, m, idx);
  const bool bnd = is_boundary<D>(idx, m);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    Ft[i * D + a] = bnd ? 0.0 : F[i * D + a];
    dUA[i * D + a] = 0.0;
  }
  const int64_t ip = (int64_t)D * n + i;
  if (active[i]) {
    dUA[ip] = phi_old[i] - phi[i];
    Ft[ip] = 0.0;
    for (int s = 0; s < NS; ++s) Kpp[(int64_t)s * n + i] = (s == center) ? 1.0 : 0.0;
    for (int s = 0; s < NS * D; ++s) Kpu[(int64_t)s * n + i] = 0.0;
    return;
  }
  dUA[ip] = 0.0;
  double f = F[ip];
  for (int s = 0; s < NS; ++s) {
    const int64_t j = neighbour<D>(idx, s, m);
    if (j < 0 || !active[j]) continue;
    f -= Kpp[(int64_t)s * n + i] * (phi_old[j] - phi[j]);
    Kpp[(int64_t)s * n + i] = 0.0;
  }
  Ft[ip] = f;
}

// y = Sinv .* (G~ x) from the assembled (reduced) stencils.
template <int D, int TB = 256>
__global__ void __launch_bounds__(TB) k_apply_assembled(MeshDev m, int64_t n,
                                                         const double* __restrict__ Kuu,
                                                         const double* __restrict__ Kpu,
                                                         const double* __restrict__ Kpp,
                                                         const double* __restrict__ x,
                                                         double* __restrict__ y,
                                                         const double* __restrict__ Sinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NS = D == 2 ? 9 : 27;
  int idx[3];
  node_index<D>(i, m, idx);
  double yu[D], yp = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) yu[a] = 0.0;
  const double* xp = x + (int64_t)D * n;
  const int64_t sy = m.nn[0], sz = (int64_t)m.nn[0] * m.nn[1];
  // branch-free over the 3^d slots: a neighbour outside the mesh is replaced by
  // node i and its x selected to zero, so all loads are independent
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = D == 3 ? s / 9 - 1 : 0;
    bool ok = (idx[0] + ox >= 0) & (idx[0] + ox < m.nn[0]) & (idx[1] + oy >= 0) &
              (idx[1] + oy < m.nn[1]);
    if (D == 3) ok = ok & (idx[2] + oz >= 0) & (idx[2] + oz < m.nn[2]);
    const int64_t j = ok ? i + ox + oy * sy + oz * sz : i;
    double xu[D];
#pragma unroll
    for (int e = 0; e < D; ++e) {
      const double v = x[j * D + e];
      xu[e] = ok ? v : 0.0;
    }
    const double vp = xp[j];
    const double xj = ok ? vp : 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int e = 0; e < D; ++e) yu[a] += Kuu[((int64_t)(s * D + a) * D + e) * n + i] * xu[e];
#pragma unroll
    for (int e = 0; e < D; ++e) yp += Kpu[(int64_t)(s * D + e) * n + i] * xu[e];
    yp += Kpp[(int64_t)s * n + i] * xj;
  }
  if (Sinv) {
#pragma unroll
    for (int a = 0; a < D; ++a) yu[a] *= Sinv[i * D + a];
    yp *= Sinv[(int64_t)D * n + i];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) y[i * D + a] = yu[a];
  y[(int64_t)D * n + i] = yp;
}

// y = Sinv .* (G~ x), matrix-free: the Section 3.1 blocks applied cell by cell
// at the quadrature points; Dirichlet / active rows are identity rows and the
// corresponding columns of x are treated as zero.
template <int D>
__global__ void __launch_bounds__(BLK) k_apply_matfree(MeshDev m, Material mat, int64_t n,
                                                       const double* __restrict__ u,
                                                       const double* __restrict__ phi,
                                                       const double* __restrict__ phit,
                                                       const uint8_t* __restrict__ active,
                                                       const double* __restrict__ x,
                                                       double* __restrict__ y,
                                                       const double* __restrict__ Sinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NA = 1 << D;
  const double wq = D == 2 ? 0.25 : 0.125;
  int idx[3];
  node_index<D>(i, m, idx);
  const bool bnd = is_boundary<D>(idx, m);
  const bool act = active[i] != 0;
  const double* xp = x + (int64_t)D * n;
  double yu[D], yp = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) yu[a] = 0.0;
  const double k1 = 1.0 - mat.kappa;
  if (!(bnd && act)) {
#pragma unroll 1
    for (int c = 0; c < NA; ++c) {
      int ci[3];
      double h[3];
      if (!adjacent_cell<D>(idx, c, m, ci, h)) continue;
      const int ai = (~c) & (NA - 1);
      double ih[D], vol = 1.0;
#pragma unroll
      for (int l = 0; l < D; ++l) {
        ih[l] = 1.0 / h[l];
        vol *= h[l];
      }
      double ue[NA][D], xe[NA][D], pe[NA], te[NA], xpe[NA];
#pragma unroll
      for (int b = 0; b < NA; ++b) {
        const int64_t nb = cell_node<D>(ci, b, m);
        const bool bb = node_on_boundary<D>(ci, b, m);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          ue[b][a] = u[nb * D + a];
          xe[b][a] = bb ? 0.0 : x[nb * D + a];
        }
        pe[b] = phi[nb];
        te[b] = phit[nb];
        xpe[b] = active[nb] ? 0.0 : xp[nb];
      }
      const double JxW = wq * vol;
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        double G[D][D], Gx[D][D], gx[D], ph = 0.0, pt = 0.0, xq = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
          gx[a] = 0.0;
#pragma unroll
          for (int l = 0; l < D; ++l) G[a][l] = Gx[a][l] = 0.0;
        }
#pragma unroll
        for (int b = 0; b < NA; ++b) {
          const double Nb = shp<D>(b, q);
          ph += Nb * pe[b];
          pt += Nb * te[b];
          xq += Nb * xpe[b];
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const double dN = dshp<D>(b, q, l) * ih[l];
            gx[l] += dN * xpe[b];
#pragma unroll
            for (int a = 0; a < D; ++a) {
              G[a][l] += ue[b][a] * dN;
              Gx[a][l] += xe[b][a] * dN;
            }
          }
        }
        double div = 0.0, divx = 0.0;
#pragma unroll
        for (int l = 0; l < D; ++l) {
          div += G[l][l];
          divx += Gx[l][l];
        }
        double sigx[D][D], sige = 0.0, sigex = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const double e = 0.5 * (G[a][l] + G[l][a]);
            const double ex = 0.5 * (Gx[a][l] + Gx[l][a]);
            const double s = 2.0 * mat.mu * e + (a == l ? mat.lam * div : 0.0);
            sigx[a][l] = 2.0 * mat.mu * ex + (a == l ? mat.lam * divx : 0.0);
            sige += s * e;
            sigex += s * ex;
          }
        const double Na = shp<D>(ai, q);
        double dNa[D];
#pragma unroll
        for (int l = 0; l < D; ++l) dNa[l] = dshp<D>(ai, q, l) * ih[l];
        if (!bnd) {
          const double wg = JxW * (k1 * pt * pt + mat.kappa);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            double t = 0.0;
#pragma unroll
            for (int l = 0; l < D; ++l) t += sigx[a][l] * dNa[l];
            yu[a] += wg * t;
          }
        }
        if (!act) {
          const double c0 = k1 * sige + 2.0 * mat.p * div + mat.Gc / mat.eps;
          double gdot = 0.0;
#pragma unroll
          for (int l = 0; l < D; ++l) gdot += gx[l] * dNa[l];
          yp += JxW * (Na * (2.0 * k1 * ph * sigex + 2.0 * mat.p * ph * divx + c0 * xq) +
                       mat.Gc * mat.eps * gdot);
        }
      }
    }
  }
  if (bnd) {
#pragma unroll
    for (int a = 0; a < D; ++a) yu[a] = x[i * D + a];
  }
  if (act) yp = xp[i];
  if (Sinv) {
#pragma unroll
    for (int a = 0; a < D; ++a) yu[a] *= Sinv[i * D + a];
    yp *= Sinv[(int64_t)D * n + i];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) y[i * D + a] = yu[a];
  y[(int64_t)D * n + i] = yp;
}

// ------------------------------------------------------------- active set ---
__global__ void k_active_set(int64_t n, int dim, const double* __restrict__ F,
                             const double* __restrict__ mass, const double* __restrict__ phi,
                             const double* __restrict__ phi_old, double c, double tau,
                             double band, int have_prev, int lock_after, uint8_t* __restrict__ raw_prev,
                             int* __restrict__ toggles, uint8_t* __restrict__ locked,
                             uint8_t* __restrict__ active, double* __restrict__ indicator,
                             int* __restrict__ counters) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool A = false, changed = false, significant = false;
  if (i < n) {
    const double ind = F[(int64_t)dim * n + i] / mass[i] + c * (phi[i] - phi_old[i]);
    const bool raw = ind > tau;
    bool lk = false;
    if (have_prev) {
      const int tg = toggles[i] + (raw != (raw_prev[i] != 0));
      toggles[i] = tg;
      lk = locked[i] || tg >= lock_after;
      locked[i] = lk;
      A = raw || lk;
      changed = A != (active[i] != 0);
      significant = changed && fabs(ind) > band;
    } else {
      toggles[i] = 0;
      locked[i] = 0;
      A = raw;
    }
    raw_prev[i] = raw;
    active[i] = A;
    if (indicator) indicator[i] = ind;
  }
  const unsigned na = __ballot_sync(0xffffffffu, A);
  const unsigned nc = __ballot_sync(0xffffffffu, changed);
  const unsigned ns = __ballot_sync(0xffffffffu, significant);
  const unsigned nl = __ballot_sync(0xffffffffu, i < n && locked[i]);
  if ((threadIdx.x & 31) == 0) {
    if (na) atomicAdd(&counters[0], __popc(na));
    if (nc) atomicAdd(&counters[1], __popc(nc));
    if (ns) atomicAdd(&counters[2], __popc(ns));
    if (nl) atomicAdd(&counters[3], __popc(nl));
  }
}

// rho_i = F_i / S_i on free rows (not Dirichlet, not active), 0 elsewhere
template <int D>
__global__ void k_scaled_reduced(MeshDev m, int64_t n, const double* __restrict__ F,
                                 const double* __restrict__ Sinv,
                                 const uint8_t* __restrict__ active, double* __restrict__ rho) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int idx[3];
  node_index<D>(i, m, idx);
  const bool bnd = is_boundary<D>(idx, m);
#pragma unroll
  for (int a = 0; a < D; ++a) rho[i * D + a] = bnd ? 0.0 : F[i * D + a] * Sinv[i * D + a];
  const int64_t ip = (int64_t)D * n + i;
  rho[ip] = active[i] ? 0.0 : F[ip] * Sinv[ip];
}

// ------------------------------------------------------------ BSR helpers ---
template <int D>
__global__ void k_stencil_count(MeshDev m, int64_t n, int* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NS = D == 2 ? 9 : 27;
  int idx[3];
  node_index<D>(i, m, idx);
  int k = 0;
  for (int s = 0; s < NS; ++s) k += neighbour<D>(idx, s, m) >= 0;
  cnt[i] = k;
}

template <int D>
__global__ void k_stencil_cols(MeshDev m, int64_t n, const int* __restrict__ rowptr,
                               int* __restrict__ col) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NS = D == 2 ? 9 : 27;
  int idx[3];
  node_index<D>(i, m, idx);
  int k = rowptr[i];
  for (int s = 0; s < NS; ++s) {
    const int64_t j = neighbour<D>(idx, s, m);
    if (j >= 0) col[k++] = (int)j;
  }
}

template <int D>
__global__ void k_stencil_vals(MeshDev m, int64_t n, int b, const double* __restrict__ K,
                               const int* __restrict__ rowptr, double* __restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NS = D == 2 ? 9 : 27;
  int idx[3];
  node_index<D>(i, m, idx);
  int64_t k = rowptr[i];
  const int bb = b * b;
  for (int s = 0; s < NS; ++s) {
    if (neighbour<D>(idx, s, m) < 0) continue;
    for (int e = 0; e < bb; ++e) val[k * bb + e] = K[((int64_t)s * bb + e) * n + i];
    ++k;
  }
}

template <int D>
__global__ void k_rigid_modes(MeshDev m, int64_t n, double* __restrict__ B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int idx[3];
  node_index<D>(i, m, idx);
  double x[3] = {0, 0, 0};
  for (int l = 0; l < D; ++l) x[l] = m.X[l][idx[l]];
  const int64_t ld = (int64_t)n * D;
  constexpr int NNS = D == 2 ? 3 : 6;
  double v[NNS][D];
  for (int k = 0; k < NNS; ++k)
    for (int a = 0; a < D; ++a) v[k][a] = 0.0;
  for (int a = 0; a < D; ++a) v[a][a] = 1.0;
  if (D == 2) {
    v[2][0] = -x[1];
    v[2][1] = x[0];
  } else {
    v[3][0] = -x[1];
    v[3][1] = x[0];
    v[4][1] = -x[2];
    v[4][2] = x[1];
    v[5][0] = x[2];
    v[5][2] = -x[0];
  }
  for (int k = 0; k < NNS; ++k)
    for (int a = 0; a < D; ++a) B[k * ld + i * D + a] = v[k][a];
}

__global__ void k_d2f(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

template <int D>
__global__ void k_node_coords(MeshDev m, int64_t n, double* __restrict__ xyz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int idx[3];
  node_index<D>(i, m, idx);
  for (int l = 0; l < D; ++l) xyz[i * D + l] = m.X[l][idx[l]];
}

// -------------------------------------------------------------- functionals --
template <int D>
__global__ void k_tcv(MeshDev m, int64_t ncell, const double* __restrict__ u,
                      const double* __restrict__ phi, double* __restrict__ partials) {
  constexpr int NA = 1 << D;
  const double wq = D == 2 ? 0.25 : 0.125;
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int ci[3];
    ci[0] = (int)(c % m.nc[0]);
    const int64_t r = c / m.nc[0];
    if (D == 2) {
      ci[1] = (int)r;
    } else {
      ci[1] = (int)(r % m.nc[1]);
      ci[2] = (int)(r / m.nc[1]);
    }
    double h[D], vol = 1.0;
    for (int l = 0; l < D; ++l) {
      h[l] = m.X[l][ci[l] + 1] - m.X[l][ci[l]];
      vol *= h[l];
    }
    double ue[NA][D], pe[NA];
#pragma unroll
    for (int b = 0; b < NA; ++b) {
      const int64_t nb = cell_node<D>(ci, b, m);
      for (int a = 0; a < D; ++a) ue[b][a] = u[nb * D + a];
      pe[b] = phi[nb];
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      double uq[D], gp[D];
      for (int a = 0; a < D; ++a) uq[a] = gp[a] = 0.0;
#pragma unroll
      for (int b = 0; b < NA; ++b) {
        const double Nb = shp<D>(b, q);
        for (int a = 0; a < D; ++a) {
          uq[a] += Nb * ue[b][a];
          gp[a] += dshp<D>(b, q, a) / h[a] * pe[b];
        }
      }
      double dot = 0.0;
      for (int a = 0; a < D; ++a) dot += uq[a] * gp[a];
      s += dot;
    }
    acc += wq * vol * s;
  }
  // block reduction (fixed order)
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int np, double* __restrict__ out) {
  __shared__ double sh[256];
  double a = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) a += partials[k];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// COD: block per (column, point) entry; threads walk the cells along the last axis
template <int D>
__global__ void k_cod(MeshDev m, const CodColumn* __restrict__ cols, const double* __restrict__ u,
                      const double* __restrict__ phi, double* __restrict__ out) {
  const CodColumn cc = cols[blockIdx.x];
  constexpr int NA = 1 << D;
  constexpr int L = D - 1;   // integration axis
  double acc = 0.0;
  for (int j = threadIdx.x; j < m.nc[L]; j += blockDim.x) {
    int ci[3];
    double loc[3], h[3];
    for (int a = 0; a < L; ++a) {
      ci[a] = cc.col[a];
      loc[a] = cc.xi[a];
    }
    ci[L] = j;
    for (int l = 0; l < D; ++l) h[l] = m.X[l][ci[l] + 1] - m.X[l][ci[l]];
    double ue[NA][D], pe[NA];
    for (int b = 0; b < NA; ++b) {
      const int64_t nb = cell_node<D>(ci, b, m);
      for (int a = 0; a < D; ++a) ue[b][a] = u[nb * D + a];
      pe[b] = phi[nb];
    }
    for (int g = 0; g < 2; ++g) {
      loc[L] = gauss_pt(g);
      double uq[D], gp[D];
      for (int a = 0; a < D; ++a) uq[a] = gp[a] = 0.0;
      for (int b = 0; b < NA; ++b) {
        double f[D];
        for (int l = 0; l < D; ++l) f[l] = ((b >> l) & 1) ? loc[l] : 1.0 - loc[l];
        double Nb = 1.0;
        for (int l = 0; l < D; ++l) Nb *= f[l];
        for (int a = 0; a < D; ++a) uq[a] += Nb * ue[b][a];
        for (int l = 0; l < D; ++l) {
          double d = ((b >> l) & 1) ? 1.0 : -1.0;
          for (int k = 0; k < D; ++k)
            if (k != l) d *= f[k];
          gp[l] += d / h[l] * pe[b];
        }
      }
      double dot = 0.0;
      for (int a = 0; a < D; ++a) dot += uq[a] * gp[a];
      acc += 0.5 * h[L] * dot;
    }
  }
  __shared__ double sh[128];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = cc.w * sh[0];
}

}  // namespace

// ----------------------------------------------------------------- launchers --
#define DISPATCH(dim, ...) \
  do {                     \
    if ((dim) == 2) {      \
      constexpr int D = 2; \
      __VA_ARGS__;         \
    } else {               \
      constexpr int D = 3; \
      __VA_ARGS__;         \
    }                      \
  } while (0)

namespace {
constexpr double B8 = 8.0;
inline double NSd(int d) { return d == 2 ? 9.0 : 27.0; }
}  // namespace

// ------------------------------------------------------ element-tile autotune --
// The FP64 element kernels compute one node or one cell per thread with no
// cross-thread sums, so their block size ("tile") changes only speed, never a
// result.  Each is compiled for 64, 128 and 256 threads per block (launch bounds
// to match); at its first use for a given dimension and size class (power of
// two of the thread count), outside any stream capture, every tile is timed on
// the call's own data and the fastest is kept for the process.  PFF_ELEM_TILE =
// 64 | 128 | 256 forces one tile.
namespace {
constexpr int kTiles[3] = {64, 128, 256};
enum TileKernel { TK_RESID_QP, TK_RESID_GATHER, TK_ASM_UU, TK_ASM_PHI_QP, TK_ASM_PHI_GATHER, TK_APPLY };
const char* const kTileKernelNames[] = {"residual_qp", "residual_gather", "assemble_uu",
                                        "assemble_phi_qp", "assemble_phi_gather", "apply_assembled"};
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int>, int> g_tile_best;   // (kernel, dim, size class) -> tile index

int forced_tile() {
  static const int f = [] {
    const char* e = std::getenv("PFF_ELEM_TILE");
    if (!e) return -1;
    const int v = std::atoi(e);
    for (int t = 0; t < 3; ++t)
      if (kTiles[t] == v) return t;
    return -1;
  }();
  return f;
}

// tile index for kernel k over n threads; `launch(t)` launches it with tile t
template <class F>
int pick_tile(TileKernel k, int dim, int64_t n, int def, cudaStream_t s, F&& launch) {
  const int f = forced_tile();
  if (f >= 0) return f;
  int cls = 0;
  while (cls < 62 && (int64_t(1) << (cls + 1)) <= n) ++cls;
  const auto key = std::make_tuple((int)k, dim, cls);
  {
    std::lock_guard<std::mutex> g(g_tile_mu);
    auto it = g_tile_best.find(key);
    if (it != g_tile_best.end()) return it->second;
  }
  char rkey[96];
  std::snprintf(rkey, sizeof(rkey), "tile:%s:%d:%d", kTileKernelNames[k], dim, cls);
  int recorded = 0;
  if (tune_lookup(rkey, &recorded) && recorded >= 0 && recorded < 3) {
    std::lock_guard<std::mutex> g(g_tile_mu);
    g_tile_best[key] = recorded;
    return recorded;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return def;   // no timing inside a capture; decided at the next uncaptured call
  }
  cudaEvent_t a, b;
  PFF_CUDA(cudaEventCreate(&a));
  PFF_CUDA(cudaEventCreate(&b));
  int best = def;
  float best_ms = 1e30f;
  for (int t = 0; t < 3; ++t) {
    launch(t);   // warm
    PFF_CUDA(cudaEventRecord(a, s));
    launch(t);
    launch(t);
    PFF_CUDA(cudaEventRecord(b, s));
    PFF_CUDA(cudaEventSynchronize(b));
    PFF_LAUNCH("element tile tuning");
    float ms = 0.f;
    PFF_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (verbose())
      std::fprintf(stderr, "[pff] tile tune %s %dd n=%lld tile %d: %.2f us\n", kTileKernelNames[k], dim,
                   (long long)n, kTiles[t], 500.0f * ms);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  count_launch(9);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  tune_store(rkey, best);
  std::lock_guard<std::mutex> g(g_tile_mu);
  g_tile_best[key] = best;
  return best;
}
}  // namespace

#define TILE_DISPATCH(t, ...)         \
  do {                                \
    if ((t) == 0) {                   \
      constexpr int TB = kTiles[0];   \
      __VA_ARGS__;                    \
    } else if ((t) == 1) {            \
      constexpr int TB = kTiles[1];   \
      __VA_ARGS__;                    \
    } else {                          \
      constexpr int TB = kTiles[2];   \
      __VA_ARGS__;                    \
    }                                 \
  } while (0)

// launch kernel K (template <int D, int TB>) over `count` threads with its tuned tile
#define TUNED_LAUNCH(kind, count, def, K, ...)                                                  \
  do {                                                                                        \
    auto launch_ = [&](int t_) {                                                              \
      TILE_DISPATCH(t_, DISPATCH(m.dim, (K<D, TB><<<grid_for((count), TB), TB, 0, s>>>(__VA_ARGS__)))); \
    };                                                                                        \
    launch_(pick_tile(kind, m.dim, (count), (def), s, launch_));                              \
  } while (0)

void launch_phi_tilde(const MeshDev& /*m*/, int64_t n, int steps_done, const double* phi_old,
                      const double* phi_prev, double* phit, cudaStream_t s) {
  ProfScope ps("phi_tilde", 3.0 * B8 * n, s);
  // extrapolation needs two computed time levels: the initial crack field is not one
  k_phi_tilde<<<grid_for(n, 256), 256, 0, s>>>(n, steps_done <= 1, phi_old, phi_prev, phit);
  PFF_LAUNCH("phi_tilde");
}

void launch_lumped_mass(const MeshDev& m, int64_t n, double* mass, cudaStream_t s) {
  Material dummy{1, 0, 1, 0, 1, 0, 0, 0};
  ProfScope ps("lumped_mass", B8 * n, s);
  DISPATCH(m.dim, (k_mass_and_sphi<D><<<grid_for(n, BLK), BLK, 0, s>>>(m, dummy, n, mass, nullptr)));
  PFF_LAUNCH("lumped_mass");
}

int64_t qp_doubles(int dim, int64_t n_cells) {
  const int na = 1 << dim;
  const int rec = dim == 2 ? res_rec<2>() : res_rec<3>();   // the larger of the two records
  static_assert(res_rec<2>() >= phi_rec<2>() && res_rec<3>() >= phi_rec<3>(), "record sizes");
  return (int64_t)na * rec * n_cells;
}

void launch_residual(const MeshDev& m, const Material& mat, int64_t n, int64_t n_cells,
                     const double* u, const double* phi, const double* phit, double* qp,
                     double* F, cudaStream_t s) {
  // reads u, phi, phi~; writes F (the quadrature records stay in L2 / are not counted)
  ProfScope ps("residual", B8 * n * (2.0 * m.dim + 3.0), s, 2);
  TUNED_LAUNCH(TK_RESID_QP, n_cells, 1, k_residual_qp, m, mat, n_cells, u, phi, phit, qp);
  TUNED_LAUNCH(TK_RESID_GATHER, n, 1, k_residual_gather, m, n, n_cells, qp, F);
  PFF_LAUNCH("residual");
}

void launch_assemble_uu(const MeshDev& m, const Material& mat, int64_t n, const double* phit,
                        double* Kuu, cudaStream_t s) {
  ProfScope ps("assemble_uu", B8 * n * (1.0 + NSd(m.dim) * m.dim * m.dim), s);
  TUNED_LAUNCH(TK_ASM_UU, n, 1, k_assemble_uu, m, mat, n, phit, Kuu);
  PFF_LAUNCH("assemble_uu");
}

void launch_assemble_phi(const MeshDev& m, const Material& mat, int64_t n, int64_t n_cells,
                         const double* u, const double* phi, double* qp, double* Kpu, double* Kpp,
                         cudaStream_t s) {
  ProfScope ps("assemble_phi", B8 * n * ((m.dim + 1.0) + NSd(m.dim) * (m.dim + 1.0)), s, 2);
  TUNED_LAUNCH(TK_ASM_PHI_QP, n_cells, 1, k_assemble_phi_qp, m, mat, n_cells, u, phi, qp);
  TUNED_LAUNCH(TK_ASM_PHI_GATHER, n, 1, k_assemble_phi_gather, m, mat, n, n_cells, qp, Kpu, Kpp);
  PFF_LAUNCH("assemble_phi");
}

void launch_scaling(const MeshDev& m, const Material& mat, int64_t n, const double* Kuu,
                    double* S, double* Sinv, cudaStream_t s) {
  const int d = m.dim;
  ProfScope ps("scaling", B8 * n * (3.0 * d + 3.0), s, 3);
  DISPATCH(d, (k_scaling_u<D><<<grid_for(n, 256), 256, 0, s>>>(n, Kuu, S, Sinv)));
  DISPATCH(d, (k_mass_and_sphi<D><<<grid_for(n, BLK), BLK, 0, s>>>(m, mat, n, nullptr,
                                                                    S + (int64_t)d * n)));
  k_invert<<<grid_for(n, 256), 256, 0, s>>>(n, S + (int64_t)d * n, Sinv + (int64_t)d * n);
  PFF_LAUNCH("scaling");
}

void launch_reduce_phi(const MeshDev& m, int64_t n, const uint8_t* active, const double* phi,
                       const double* phi_old, const double* F, double* Ft, double* dUA,
                       double* Kpu, double* Kpp, cudaStream_t s) {
  // reads F, phi, phi_old, active, Kpp; writes Ft, dUA, Kpp (masked)
  ProfScope ps("reduce_phi", n * (B8 * (3.0 * (m.dim + 1) + 2.0 + 2.0 * NSd(m.dim)) + 1.0), s);
  DISPATCH(m.dim, (k_reduce_phi<D><<<grid_for(n, 256), 256, 0, s>>>(m, n, active, phi, phi_old, F,
                                                                     Ft, dUA, Kpu, Kpp)));
  PFF_LAUNCH("reduce_phi");
}

void launch_apply_assembled(const MeshDev& m, const int64_t n, const double* Kuu, const double* Kpu,
                            const double* Kpp, const double* x, double* y, const double* Sinv,
                            cudaStream_t s) {
  // stencils (d^2 + d + 1 values per slot), x, y, Sinv
  const double per = NSd(m.dim) * (m.dim * m.dim + m.dim + 1.0) + (m.dim + 1.0) * (Sinv ? 3.0 : 2.0);
  ProfScope ps("apply_assembled", B8 * n * per, s);
  TUNED_LAUNCH(TK_APPLY, n, 2, k_apply_assembled, m, n, Kuu, Kpu, Kpp, x, y, Sinv);
  PFF_LAUNCH("apply_assembled");
}

void launch_apply_matfree(const MeshDev& m, const Material& mat, int64_t n, const double* u,
                          const double* phi, const double* phit, const uint8_t* active,
                          const double* x, double* y, const double* Sinv, cudaStream_t s) {
  // u, phi, phi~, active, x, y, Sinv
  const double per = B8 * (m.dim + 2.0 + (m.dim + 1.0) * (Sinv ? 3.0 : 2.0)) + 1.0;
  ProfScope ps("apply_matfree", n * per, s);
  DISPATCH(m.dim, (k_apply_matfree<D><<<grid_for(n, BLK), BLK, 0, s>>>(m, mat, n, u, phi, phit,
                                                                       active, x, y, Sinv)));
  PFF_LAUNCH("apply_matfree");
}

void launch_active_set(int64_t n, int dim, const double* F, const double* mass, const double* phi,
                       const double* phi_old, double c, double tau, double band, int have_prev,
                       int lock_after,
                       uint8_t* raw_prev, int* toggles, uint8_t* locked, uint8_t* active,
                       double* indicator, int* counters, cudaStream_t s) {
  PFF_CUDA(cudaMemsetAsync(counters, 0, 4 * sizeof(int), s));
  ProfScope ps("active_set", n * (B8 * (indicator ? 5.0 : 4.0) + 14.0), s);
  k_active_set<<<grid_for(n, 256), 256, 0, s>>>(n, dim, F, mass, phi, phi_old, c, tau, band, have_prev,
                                                lock_after, raw_prev, toggles, locked, active,
                                                indicator, counters);
  PFF_LAUNCH("active_set");
}

void launch_scaled_reduced(const MeshDev& m, int64_t n, const double* F, const double* Sinv,
                           const uint8_t* active, double* rho, cudaStream_t s) {
  ProfScope ps("scaled_reduced", n * (B8 * 3.0 * (m.dim + 1.0) + 1.0), s);
  DISPATCH(m.dim, (k_scaled_reduced<D><<<grid_for(n, 256), 256, 0, s>>>(m, n, F, Sinv, active, rho)));
  PFF_LAUNCH("scaled_reduced");
}

void build_stencil_bsr_structure(const MeshDev& m, int64_t n, int b, Bsr& A, cudaStream_t s) {
  A.nrows = A.ncols = (int)n;
  A.br = A.bc = b;
  A.rowptr = dalloc<int>(n + 1);
  int* cnt = dalloc<int>(n + 1);
  count_launch();
  DISPATCH(m.dim, (k_stencil_count<D><<<grid_for(n, 256), 256, 0, s>>>(m, n, cnt)));
  PFF_LAUNCH("stencil_count");
  int total = 0;
  exclusive_scan_int(cnt, A.rowptr, (int)n, &total, s);
  A.nnzb = total;
  A.col = dalloc<int>(total);
  A.val = dalloc<double>((size_t)total * b * b);
  count_launch();
  DISPATCH(m.dim, (k_stencil_cols<D><<<grid_for(n, 256), 256, 0, s>>>(m, n, A.rowptr, A.col)));
  PFF_LAUNCH("stencil_cols");
  PFF_CUDA(cudaStreamSynchronize(s));
  dfree(cnt);
}

void launch_stencil_to_bsr(const MeshDev& m, int64_t n, int b, const double* K, const Bsr& A,
                           cudaStream_t s) {
  ProfScope ps("stencil_to_bsr", 2.0 * B8 * A.nnzb * b * b + 4.0 * n, s);
  DISPATCH(m.dim, (k_stencil_vals<D><<<grid_for(n, 256), 256, 0, s>>>(m, n, b, K, A.rowptr, A.val)));
  PFF_LAUNCH("stencil_vals");
}

void launch_rigid_modes(const MeshDev& m, int64_t n, double* B, cudaStream_t s) {
  count_launch();
  DISPATCH(m.dim, (k_rigid_modes<D><<<grid_for(n, 256), 256, 0, s>>>(m, n, B)));
  PFF_LAUNCH("rigid_modes");
}

void convert_d2f(const double* a, float* b, int64_t n, cudaStream_t s) {
  ProfScope ps("to_f32", 12.0 * n, s);
  k_d2f<<<grid_for(n, 256), 256, 0, s>>>(n, a, b);
  PFF_LAUNCH("d2f");
}

void launch_node_coords(const MeshDev& m, int64_t n, double* xyz, cudaStream_t s) {
  count_launch();
  DISPATCH(m.dim, (k_node_coords<D><<<grid_for(n, 256), 256, 0, s>>>(m, n, xyz)));
  PFF_LAUNCH("node_coords");
}

void tcv_dev(const MeshDev& m, int64_t n_cells, const double* u, const double* phi, double* out,
             double* partials, cudaStream_t s) {
  const int nb = (int)std::min<int64_t>(RED_PARTIALS, (n_cells + 255) / 256);
  ProfScope ps("tcv", B8 * n_cells * (m.dim + 1.0), s, 2);
  DISPATCH(m.dim, (k_tcv<D><<<nb, 256, 0, s>>>(m, n_cells, u, phi, partials)));
  k_sum_partials<<<1, 256, 0, s>>>(partials, nb, out);
  PFF_LAUNCH("tcv");
}

void cod_dev(const MeshDev& m, const CodColumn* cols, int ncols, const double* u, const double* phi,
             double* out, int /*npts*/, cudaStream_t s) {
  if (ncols == 0) return;
  ProfScope ps("cod", 0.0, s);
  DISPATCH(m.dim, (k_cod<D><<<ncols, 128, 0, s>>>(m, cols, u, phi, out)));
  PFF_LAUNCH("cod");
}

}  // namespace pff
