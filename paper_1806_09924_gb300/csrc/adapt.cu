// Adaptive refinement of the tensor-product mesh (Section 3, refinement
// strategy): the gradient-jump indicator of the displacements per cell, its
// sums over axis slabs together with the slab's smallest phase-field value,
// and the Q1 transfer of nodal fields onto a refined mesh.
//
// Indicator (Kelly-type gradient jump): eta_K^2 = (h_K / 24) * sum over the
// interior faces F of K of the integral over F of |[du/dn]|^2, h_K the cell
// diameter.  On a Q1 field the normal derivative across a face normal to axis
// a is the nodal difference quotient of the cell on either side, interpolated
// multilinearly over the face; its jump is therefore multilinear on the face,
// given by its corner values J_c, and the integral is exact in closed form:
// area * sum_{c,c'} J_c J_c' * prod over the face axes of (1/3 if c and c'
// share the corner coordinate, else 1/6) -- the Q1 face mass matrix.
#include "pff_internal.h"

namespace pff {

namespace {

template <int D>
__global__ void k_jump_indicator(MeshDev m, int64_t ncell, const double* __restrict__ u,
                                 double* __restrict__ eta2) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  int ci[3] = {0, 0, 0};
  ci[0] = (int)(c % m.nc[0]);
  const int64_t r = c / m.nc[0];
  if (D == 2) {
    ci[1] = (int)r;
  } else {
    ci[1] = (int)(r % m.nc[1]);
    ci[2] = (int)(r / m.nc[1]);
  }
  double h[D], diam2 = 0.0;
#pragma unroll
  for (int l = 0; l < D; ++l) {
    h[l] = m.X[l][ci[l] + 1] - m.X[l][ci[l]];
    diam2 += h[l] * h[l];
  }
  const int64_t stride[3] = {1, m.nn[0], (int64_t)m.nn[0] * m.nn[1]};
  double total = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int o1 = (a + 1) % D, o2 = (a + 2) % D;   // face axes (o2 unused in 2d)
    double area = h[o1];
    if (D == 3) area *= h[o2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      // nodes b, b+1, b+2 along a; the face lies at b+1
      const int b = side == 0 ? ci[a] - 1 : ci[a];
      if (b < 0 || b + 2 > m.nc[a]) continue;   // boundary face
      const double hlo = m.X[a][b + 1] - m.X[a][b];
      const double hhi = m.X[a][b + 2] - m.X[a][b + 1];
      constexpr int NC = 1 << (D - 1);
      double J[NC][D];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        int64_t base = (int64_t)b * stride[a] + (int64_t)(ci[o1] + (k & 1)) * stride[o1];
        if (D == 3) base += (int64_t)(ci[o2] + ((k >> 1) & 1)) * stride[o2];
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const double u0 = u[base * D + l];
          const double u1 = u[(base + stride[a]) * D + l];
          const double u2 = u[(base + 2 * stride[a]) * D + l];
          J[k][l] = (u2 - u1) / hhi - (u1 - u0) / hlo;
        }
      }
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NC; ++k)
#pragma unroll
        for (int k2 = 0; k2 < NC; ++k2) {
          double w = ((k ^ k2) & 1) ? 1.0 / 6.0 : 1.0 / 3.0;
          if (D == 3) w *= ((k ^ k2) & 2) ? 1.0 / 6.0 : 1.0 / 3.0;
          double dot = 0.0;
#pragma unroll
          for (int l = 0; l < D; ++l) dot += J[k][l] * J[k2][l];
          s += w * dot;
        }
      total += area * s;
    }
  }
  eta2[c] = sqrt(diam2) / 24.0 * total;
}

// One block per slab (axis a, interval i), slabs of all axes numbered
// consecutively: the sum of eta2 over the slab's cells and the smallest phi
// over its nodes (a-index i or i + 1).  Fixed per-thread order and a fixed
// tree: the sums are reproducible run to run.
template <int D>
__global__ void k_slab_reduce(MeshDev m, const double* __restrict__ eta2,
                              const double* __restrict__ phi, double* __restrict__ S,
                              double* __restrict__ minphi) {
  __shared__ double ss[256], sm[256];
  int slab = blockIdx.x, a = 0;
  while (a < D - 1 && slab >= m.nc[a]) {
    slab -= m.nc[a];
    ++a;
  }
  const int i = slab;
  const int o1 = (a + 1) % D, o2 = (a + 2) % D;
  const int64_t cstride[3] = {1, m.nc[0], (int64_t)m.nc[0] * m.nc[1]};
  const int64_t nstride[3] = {1, m.nn[0], (int64_t)m.nn[0] * m.nn[1]};
  const int64_t ncells = (int64_t)m.nc[o1] * (D == 3 ? m.nc[o2] : 1);
  const int64_t nnodes = (int64_t)m.nn[o1] * (D == 3 ? m.nn[o2] : 1);
  double sum = 0.0, mn = INFINITY;
  for (int64_t p = threadIdx.x; p < ncells; p += blockDim.x) {
    const int64_t p1 = p % m.nc[o1], p2 = p / m.nc[o1];
    sum += eta2[(int64_t)i * cstride[a] + p1 * cstride[o1] + (D == 3 ? p2 * cstride[o2] : 0)];
  }
  for (int64_t p = threadIdx.x; p < nnodes; p += blockDim.x) {
    const int64_t p1 = p % m.nn[o1], p2 = p / m.nn[o1];
    const int64_t base = (int64_t)i * nstride[a] + p1 * nstride[o1] + (D == 3 ? p2 * nstride[o2] : 0);
    mn = fmin(mn, fmin(phi[base], phi[base + nstride[a]]));
  }
  ss[threadIdx.x] = sum;
  sm[threadIdx.x] = mn;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ss[threadIdx.x] += ss[threadIdx.x + w];
      sm[threadIdx.x] = fmin(sm[threadIdx.x], sm[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    S[blockIdx.x] = ss[0];
    minphi[blockIdx.x] = sm[0];
  }
}

// Q1 interpolation of a nodal field (ncomp values per node) onto the nodes of
// another tensor-product mesh: per axis, the new coordinate's source interval
// cell[a][k] and local coordinate t[a][k] (host-computed); the value is the
// sum over the 2^D source corners, in corner order, of prod_a (t or 1 - t)
// times the corner value, every product and sum rounded on its own (no fused
// multiply-add), so the result is reproducible on any FP64 implementation.
struct TransferAxes {
  const int* cell[3];
  const double* t[3];
};

template <int D>
__global__ void k_transfer(int dn0, int dn1, int64_t dn, int sn0, int sn1, TransferAxes ax,
                           const double* __restrict__ src, int ncomp, double* __restrict__ dst) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= dn) return;
  int idx[3];
  idx[0] = (int)(k % dn0);
  const int64_t r = k / dn0;
  if (D == 2) {
    idx[1] = (int)r;
  } else {
    idx[1] = (int)(r % dn1);
    idx[2] = (int)(r / dn1);
  }
  int c[3];
  double t[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    c[a] = ax.cell[a][idx[a]];
    t[a] = ax.t[a][idx[a]];
  }
  for (int comp = 0; comp < ncomp; ++comp) {
    double acc = 0.0;
#pragma unroll
    for (int corner = 0; corner < (1 << D); ++corner) {
      double w = 1.0;
      int64_t s = 0, mul = 1;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int off = (corner >> a) & 1;
        w = __dmul_rn(w, off ? t[a] : __dsub_rn(1.0, t[a]));
        s += (int64_t)(c[a] + off) * mul;
        mul *= a == 0 ? sn0 : sn1;
      }
      acc = __dadd_rn(acc, __dmul_rn(w, src[s * ncomp + comp]));
    }
    dst[k * ncomp + comp] = acc;
  }
}

#define DISPATCH_D(dim, ...) \
  do {                       \
    if ((dim) == 2) {        \
      constexpr int D = 2;   \
      __VA_ARGS__;           \
    } else {                 \
      constexpr int D = 3;   \
      __VA_ARGS__;           \
    }                        \
  } while (0)

}  // namespace

void jump_indicator_dev(const MeshDev& m, int64_t n_cells, const double* u, double* eta2,
                        cudaStream_t s) {
  if (n_cells == 0) return;
  // u is read by the 2d faces of every cell, mostly from cache: count it once
  ProfScope ps("jump_indicator", 8.0 * (n_cells + (double)m.nn[0] * m.nn[1] * (m.dim == 3 ? m.nn[2] : 1) * m.dim), s);
  DISPATCH_D(m.dim, (k_jump_indicator<D><<<grid_for(n_cells, 128), 128, 0, s>>>(m, n_cells, u, eta2)));
  PFF_LAUNCH("jump_indicator");
}

void slab_reduce_dev(const MeshDev& m, const double* eta2, const double* phi, double* S,
                     double* minphi, cudaStream_t s) {
  int slabs = 0;
  for (int a = 0; a < m.dim; ++a) slabs += m.nc[a];
  ProfScope ps("slab_reduce", 0.0, s);
  DISPATCH_D(m.dim, (k_slab_reduce<D><<<slabs, 256, 0, s>>>(m, eta2, phi, S, minphi)));
  PFF_LAUNCH("slab_reduce");
}

void transfer_dev(int dim, const int* dst_nn, const int* src_nn, const int* const* cell,
                  const double* const* t, const double* src, int ncomp, double* dst,
                  cudaStream_t s) {
  int64_t dn = 1;
  for (int a = 0; a < dim; ++a) dn *= dst_nn[a];
  if (dn == 0) return;
  TransferAxes ax{};
  for (int a = 0; a < dim; ++a) {
    ax.cell[a] = cell[a];
    ax.t[a] = t[a];
  }
  ProfScope ps("transfer", 8.0 * ncomp * dn * 2.0, s);
  DISPATCH_D(dim, (k_transfer<D><<<grid_for(dn, 256), 256, 0, s>>>(
                      dst_nn[0], dst_nn[1], dn, src_nn[0], src_nn[1], ax, src, ncomp, dst)));
  PFF_LAUNCH("transfer");
}

}  // namespace pff
