// FGMRES with the block-diagonal preconditioner of Section 3.1 and the combined
// semi-smooth Newton / primal-dual active-set loop of Section 3 (the algorithm
// the paper prints in LaTeX comments), orchestrated from the host; every vector
// operation runs in the kernels of fe_kernels.cu, linalg.cu and amg.cu.
//
// Newton iteration k of a loading step:
//   1. F = -r(U^k)                                 (residual kernel)
//   2. A_k = {i : F_phi,i/m_i + c(phi_i - phi_old,i) > tau}, plus indices
//      locked after `cycle_lock` membership changes (active-set kernel); c and
//      the printed rule's threshold tau are given in units of G_c/eps
//   3. stop if k > 0, A_k = A_{k-1}, the scaled reduced residual fell by
//      tol_newton (or below atol_newton) and the previous step was below tol_step
//   4. assemble M_phi_u, M_phi_phi (M_uu once per loading step), eliminate the
//      Dirichlet / active rows and columns (active entries get
//      delta phi = phi_old - phi, moved to the right-hand side)
//   5. FGMRES on the Jacobi-scaled reduced system S^-1 G~ dU = S^-1 F~ with the
//      right preconditioner diag(V-cycle(M_uu), V-cycle(M_phi_phi)) S
//   6. line search on ||S^-1 F~||_2 (halving), update.
// S = diag(M_uu(phi~)) (+ diag G_c(M/eps + eps K) for phi) is fixed during a
// loading step, so the reduced residual norms of different iterates compare.
#include <algorithm>
#include <mutex>
#include <map>
#include <chrono>
#include <cmath>
#include <cstdio>

#include "pff_internal.h"

namespace pff {

namespace {

__global__ void k_update(int64_t n, int dim, const double* __restrict__ u,
                         const double* __restrict__ phi, const double* __restrict__ phi_old,
                         const uint8_t* __restrict__ active, const double* __restrict__ dU,
                         double omega, double* __restrict__ uo, double* __restrict__ po) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int a = 0; a < dim; ++a) uo[i * dim + a] = u[i * dim + a] + omega * dU[i * dim + a];
  const double dp = dU[(int64_t)dim * n + i];
  po[i] = (omega == 1.0 && active[i]) ? phi_old[i] : phi[i] + omega * dp;
}

__global__ void k_add(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] += a[i];
}

__global__ void k_mul(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] * b[i];
}

// w /= sqrt(*nrm2) (into dst, and its f32_view into dstf unless null: the FP32
// values the mixed Gram-Schmidt takes its coefficients from); the scale is
// computed once per block (FP64 square roots and divides are slow on this GPU)
__global__ void k_normalize(int64_t n, const double* __restrict__ w, const double* __restrict__ nrm2,
                            double* __restrict__ dst, float* __restrict__ dstf) {
  __shared__ double sc;
  if (threadIdx.x == 0) {
    const double nn = *nrm2;
    sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  }
  __syncthreads();
  const double s = sc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[i] * s;
    dst[i] = v;
    if (dstf) dstf[i] = f32_view(v);
  }
}

// c = a - b elementwise; c may alias b (each thread reads before it writes)
__global__ void k_sub(int64_t n, const double* a, const double* b, double* c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] - b[i];
}

__global__ void k_count_ties(int64_t n, const double* __restrict__ ind, double tau,
                             int* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool tie = i < n && fabs(ind[i]) <= tau;
  const unsigned b = __ballot_sync(0xffffffffu, tie);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(cnt, __popc(b));
}

// zero the phase-field rows of rho whose indicator lies in the tie band
__global__ void k_zero_ties(int64_t n, int dim, const double* __restrict__ ind, double band,
                            double* __restrict__ rho) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && fabs(ind[i]) <= band) rho[(int64_t)dim * n + i] = 0.0;
}

void launch_update(cudaStream_t s, int64_t n, int dim, const double* u, const double* phi,
                   const double* phi_old, const uint8_t* active, const double* dU, double omega,
                   double* uo, double* po) {
  ProfScope ps("update", n * (8.0 * (3.0 * dim + 4.0) + 1.0), s);
  k_update<<<grid_for(n, 256), 256, 0, s>>>(n, dim, u, phi, phi_old, active, dU, omega, uo, po);
  PFF_LAUNCH("update");
}

// Sw = S / w_block, Sinvw = w_block * Sinv (w_u on the displacement rows, w_p on the rest)
__global__ void k_block_weights(int64_t N, int64_t nu, const double* __restrict__ S,
                                const double* __restrict__ Sinv, double wu, double wp,
                                double* __restrict__ Sw, double* __restrict__ Sinvw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double w = i < nu ? wu : wp;
  Sw[i] = S[i] / w;
  Sinvw[i] = Sinv[i] * w;
}

void launch_block_weights(cudaStream_t s, int64_t N, int64_t nu, const double* S,
                          const double* Sinv, double wu, double wp, double* Sw, double* Sinvw) {
  ProfScope ps("block_weights", 32.0 * N, s);
  k_block_weights<<<grid_for(N, 256), 256, 0, s>>>(N, nu, S, Sinv, wu, wp, Sw, Sinvw);
  PFF_LAUNCH("block_weights");
}

void sync(pff_problem* P) { PFF_CUDA(cudaStreamSynchronize(P->stream)); }

double fetch(pff_problem* P, const double* d) {
  PFF_CUDA(cudaMemcpyAsync(P->h_scalars, d, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  return P->h_scalars[0];
}

}  // namespace

void scale_into(const double* s, const double* x, double* y, int64_t n, cudaStream_t st) {
  ProfScope ps("vec_mul", 24.0 * n, st);
  k_mul<<<grid_for(n, 256), 256, 0, st>>>(n, s, x, y);
  PFF_LAUNCH("scale");
}

void ensure_krylov(pff_problem* P, int m) {
  if (P->krylov_m >= m) return;
  dfree(P->V);
  dfree(P->Z);
  dfree(P->w);
  dfree(P->h);
  dfree(P->tmp);
  dfree(P->gs_part);
  dfree(P->Vf);
  P->Vf = nullptr;   // reallocated at the new size by the mixed path
  if (P->h_host) cudaFreeHost(P->h_host);
  const int64_t N = P->n_dofs;
  P->V = dalloc<double>((size_t)(m + 1) * N);
  P->Z = dalloc<double>((size_t)m * N);
  P->w = dalloc<double>(N);
  P->tmp = dalloc<double>(N);
  P->h = dalloc<double>(4 * (m + 2));
  P->gs_part = dalloc<float>((size_t)(m + 2) * GS_MAX_BLOCKS);
  PFF_CUDA(cudaMallocHost(&P->h_host, sizeof(double) * 4 * (m + 2)));
  P->krylov_m = m;
}

void compute_residual(pff_problem* P, const double* u, const double* phi, double* F) {
  launch_residual(P->mesh(), P->mat, P->n_nodes, P->n_cells, u, phi, P->phit, P->qp, F, P->stream);
}

void compute_active_set(pff_problem* P, double c_rel, double tol_active, double tol_change,
                        int lock_after, bool track) {
  const double scale = P->mat.Gc / P->mat.eps;   // indicator constants in units of G_c/eps
  launch_active_set(P->n_nodes, P->dim, P->F, P->mass, P->phi, P->phi_old, c_rel * scale,
                    tol_active * scale, tol_change * scale, track ? 1 : 0, lock_after, P->raw_prev, P->toggles,
                    P->locked, P->active, P->indicator, P->counters, P->stream);
}

void assemble_all(pff_problem* P) {
  const auto m = P->mesh();
  if (!P->uu_assembled) {
    launch_assemble_uu(m, P->mat, P->n_nodes, P->phit, P->Kuu, P->stream);
    launch_scaling(m, P->mat, P->n_nodes, P->Kuu, P->S, P->Sinv, P->stream);
    P->uu_assembled = true;
  }
  launch_assemble_phi(m, P->mat, P->n_nodes, P->n_cells, P->u, P->phi, P->qp, P->Kpu, P->Kpp,
                      P->stream);
  launch_reduce_phi(m, P->n_nodes, P->active, P->phi, P->phi_old, P->F, P->Ft, P->dUA, P->Kpu,
                    P->Kpp, P->stream);
  P->phi_assembled = true;
}

void apply_jacobian(pff_problem* P, int variant, const double* x, double* y, const double* Sinv) {
  if (variant == PFF_APPLY_MATFREE) {
    launch_apply_matfree(P->mesh(), P->mat, P->n_nodes, P->u, P->phi, P->phit, P->active, x, y,
                         Sinv, P->stream);
  } else {
    if (!P->phi_assembled) fail(PFF_ERR_INVALID_ARG, "assembled apply requested before assembly");
    launch_apply_assembled(P->mesh(), P->n_nodes, P->Kuu, P->Kpu, P->Kpp, x, y, Sinv, P->stream);
  }
}

__global__ void k_abs_diff(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fabs(a[i] - b[i]);
}

__global__ void k_count_diff(int64_t n, const uint8_t* __restrict__ a, const uint8_t* __restrict__ b,
                             int* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool d = i < n && a[i] != b[i];
  const unsigned m = __ballot_sync(0xffffffffu, d);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(cnt, __popc(m));
}

// number of indices where two masks differ
static int64_t count_diff(pff_problem* P, const uint8_t* a, const uint8_t* b, int64_t n) {
  count_launch();
  PFF_CUDA(cudaMemsetAsync(P->counters + 4, 0, sizeof(int), P->stream));
  k_count_diff<<<grid_for(n, 256), 256, 0, P->stream>>>(n, a, b, P->counters + 4);
  PFF_LAUNCH("count_diff");
  PFF_CUDA(cudaMemcpyAsync(P->h_counters + 4, P->counters + 4, sizeof(int), cudaMemcpyDeviceToHost,
                           P->stream));
  PFF_CUDA(cudaStreamSynchronize(P->stream));
  return P->h_counters[4];
}

// PFF_APPLY_AUTO: the assembled-stencil and the matrix-free FP64 Jacobian apply
// compute the same product; time each on this problem once (3 launches after a
// warm one, CUDA events on the problem's stream) and keep the faster.  The
// choice is remembered per (dimension, log2 node count) for later problems.
static void choose_apply(pff_problem* P) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  const auto key = std::make_pair(P->dim, (int)std::log2((double)std::max<int64_t>(1, P->n_nodes)));
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      P->apply_variant = it->second;
      P->apply_auto = false;
      return;
    }
  }
  const std::string rkey = "apply:" + std::to_string(key.first) + ":" + std::to_string(key.second);
  int recorded = 0;
  if (tune_lookup(rkey, &recorded) &&
      (recorded == PFF_APPLY_ASSEMBLED || recorded == PFF_APPLY_MATFREE)) {
    P->apply_variant = recorded;
    P->apply_auto = false;
    std::lock_guard<std::mutex> g(mu);
    cache[key] = recorded;
    return;
  }
  cudaEvent_t e0, e1;
  PFF_CUDA(cudaEventCreate(&e0));
  PFF_CUDA(cudaEventCreate(&e1));
  const double* Si = P->op_Sinv ? P->op_Sinv : P->Sinv;
  float best_ms = 1e30f;
  int best = PFF_APPLY_ASSEMBLED;
  for (int v : {PFF_APPLY_ASSEMBLED, PFF_APPLY_MATFREE}) {
    apply_jacobian(P, v, P->F, P->tmp, Si);
    PFF_CUDA(cudaEventRecord(e0, P->stream));
    for (int r = 0; r < 3; ++r) apply_jacobian(P, v, P->F, P->tmp, Si);
    PFF_CUDA(cudaEventRecord(e1, P->stream));
    PFF_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    PFF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (verbose())
      std::fprintf(stderr, "[pff] Jacobian apply %s: %.1f us\n",
                   v == PFF_APPLY_ASSEMBLED ? "assembled" : "matrix-free", 1e3 * ms / 3);
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->apply_variant = best;
  P->apply_auto = false;
  tune_store(rkey, best);
  std::lock_guard<std::mutex> g(mu);
  cache[key] = best;
}

// max_i |a_i - b_i| (device vectors of length n <= n_dofs)
static double max_abs_diff(pff_problem* P, const double* a, const double* b, int64_t n) {
  double* t = P->tmp ? P->tmp : dalloc<double>(n);
  count_launch();
  k_abs_diff<<<grid_for(n, 256), 256, 0, P->stream>>>(n, a, b, t);
  PFF_LAUNCH("abs_diff");
  nrm_inf_dev(t, n, P->d_scalars, P->partials, P->stream);
  PFF_CUDA(cudaMemcpyAsync(P->h_scalars, P->d_scalars, sizeof(double), cudaMemcpyDeviceToHost,
                           P->stream));
  PFF_CUDA(cudaStreamSynchronize(P->stream));
  if (!P->tmp) dfree(t);
  return P->h_scalars[0];
}

void precond_setup(pff_problem* P, const pff_options& o, bool allow_reuse) {
  P->precision = o.precision;
  P->overlap = o.precond_overlap != 0;
  l2_cache_bytes();   // device query made here, never inside a captured iteration
  if (o.precond == PFF_PC_JACOBI) return;
  AmgParams ap;
  ap.theta = o.amg_theta;
  ap.coarse_max = o.amg_coarse_max;
  ap.cheb_degree = o.cheb_degree;
  // -1: by dimension (measured on the graded 2d and 3d workloads)
  ap.cheb_degree_coarse = o.cheb_degree_coarse > 0    ? o.cheb_degree_coarse
                          : o.cheb_degree_coarse == 0 ? o.cheb_degree
                                                      : (P->dim == 3 ? 3 : 2);
  ap.cheb_ratio = o.cheb_ratio > 1.0 ? o.cheb_ratio : 30.0;
  ap.coords = P->xyz;
  ap.coord_dim = P->dim;
  ap.mixed = o.precision == PFF_PREC_MIXED;
  ap.spmv_group = o.spmv_group;
  const auto m = P->mesh();
  const int64_t n = P->n_nodes;
  // the finest level of each hierarchy smooths on the assembled stencil itself;
  // its FP32 copy (mixed precision) is made before a build, whose Lanczos
  // estimate of the finest level then applies the stencil too
  auto convert_stencil = [&](const double* K, float*& Kf, int b) {
    if (!ap.mixed) return;
    if (!Kf) Kf = dalloc<float>(stencil_f32_count(P->dim, b, n));
    if (P->dim == 2 && b == 2) stencil_to_node_major(K, Kf, n, P->stream);
    else stencil_to_f32(P->dim, b, K, Kf, n, P->stream);
  };
  auto with_stencil = [&](AmgParams q, const double* K, const float* Kf, int b) {
    q.mesh = m;
    q.st = K;
    q.stf = ap.mixed ? Kf : nullptr;
    q.stf_node_major = P->dim == 2 && b == 2;
    return q;
  };
  auto use_stencil = [&](Amg& amg, const double* K, const float* Kf, int b) {
    if (amg.lev.empty()) return;
    AmgLevel& L0 = amg.lev[0];
    L0.stencil = true;
    L0.mesh = m;
    L0.st = K;
    if (ap.mixed) {
      L0.stf_node_major = P->dim == 2 && b == 2;
      L0.stf = Kf;
    }
  };
  // Displacement block: M_uu depends on phi~ alone, and the aggregates on the
  // node coordinates alone.  A hierarchy carries over to the next loading step
  // while phi~ moved by at most amg_reuse_tol at every node (and for at most
  // 8 loading steps); the finest level then smooths on the new stencil with
  // its new diagonal, the coarse levels keep the Galerkin operators of the
  // build.  FGMRES is flexible, so a stale coarse space costs iterations only.
  bool reuse_u = P->amg_u_valid && P->amg_u.mixed == ap.mixed && !P->amg_u.lev.empty();
  if (reuse_u && P->amg_u_check) {
    reuse_u = o.amg_reuse != 0 && P->phit_built != nullptr && P->amg_u_age < 8;
    if (reuse_u) {
      const double dphi = max_abs_diff(P, P->phit, P->phit_built, n);
      reuse_u = dphi <= o.amg_reuse_tol;
      if (verbose())
        std::fprintf(stderr, "[pff] phi~ moved by %.3e since the displacement AMG build: %s\n",
                     dphi, reuse_u ? "reuse" : "rebuild");
    }
    if (reuse_u) {
      AmgLevel& L0 = P->amg_u.lev[0];
      launch_stencil_dinv(m, n, P->dim, P->Kuu, L0.dinv, ap.mixed ? L0.dinvf : nullptr, P->stream);
      convert_stencil(P->Kuu, P->Kuu_f, P->dim);
      use_stencil(P->amg_u, P->Kuu, P->Kuu_f, P->dim);
      P->amg_u_age += 1;
    }
    P->amg_u_check = false;
  }
  if (!reuse_u) {
    ProfScope ps("amg_setup_u", 0.0, P->stream, 0);   // wall time of the build (syncs inside)
    launch_stencil_to_bsr(m, n, P->dim, P->Kuu, P->Auu, P->stream);
    // near-null space: the rigid-body modes (translations first in Bu), or translations only
    const bool rot = o.amg_rotations < 0 ? P->dim == 2 : o.amg_rotations == 1;
    const int nns = rot ? (P->dim == 2 ? 3 : 6) : P->dim;
    convert_stencil(P->Kuu, P->Kuu_f, P->dim);
    amg_build(P->amg_u, P->Auu, P->Bu, nns, with_stencil(ap, P->Kuu, P->Kuu_f, P->dim), P->stream);
    use_stencil(P->amg_u, P->Kuu, P->Kuu_f, P->dim);
    if (!P->phit_built) P->phit_built = dalloc<double>(n);
    PFF_CUDA(cudaMemcpyAsync(P->phit_built, P->phit, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                             P->stream));
    P->amg_u_age = 0;
    P->amg_u_check = false;
    P->amg_u_valid = true;
    P->cur.amg_builds_u += 1;
  }
  // Phase-field block: rebuild when the active set differs from the one the
  // hierarchy was built for in more than amg_rebuild_phi of the nodes (also
  // across loading steps), or after amg_age_phi Newton iterations; otherwise
  // keep the hierarchy and refresh only the finest level's stencil values and
  // diagonal.  FGMRES
  // converges to its tolerance either way: a stale coarse space costs
  // iterations, not accuracy.
  bool rebuild = !allow_reuse || !P->amg_p_valid || !P->amg_p.built ||
                 P->amg_p.mixed != ap.mixed || P->phi_amg_age >= o.amg_age_phi ||
                 P->amg_p.lev.empty() || !P->active_built;
  if (!rebuild) rebuild = (double)count_diff(P, P->active, P->active_built, n) > o.amg_rebuild_phi * n;
  convert_stencil(P->Kpp, P->Kpp_f, 1);
  if (rebuild) {
    ProfScope ps("amg_setup_phi", 0.0, P->stream, 0);
    launch_stencil_to_bsr(m, n, 1, P->Kpp, P->App, P->stream);
    AmgParams app = with_stencil(ap, P->Kpp, P->Kpp_f, 1);
    // -1: smoothing only while the mass term G_c/eps M dominates the block (cells of
    // at least eps/4; the workloads here have eps = 2-4 h_min), the full hierarchy on
    // meshes refined below that (measured: a refined 32^2 cyclic-loading step past
    // the critical pressure needs it, FGMRES stalls at its cap with smoothing only)
    int levels_phi = o.amg_levels_phi;
    if (levels_phi < 0) {
      double hmin = INFINITY;
      for (int a = 0; a < P->dim; ++a)
        for (size_t i = 0; i + 1 < P->hX[a].size(); ++i) hmin = std::min(hmin, P->hX[a][i + 1] - P->hX[a][i]);
      levels_phi = hmin >= 0.25 * P->mat.eps ? 1 : 0;
    }
    if (levels_phi > 0) app.max_levels = levels_phi - 1;
    if (o.cheb_degree_phi > 0) app.cheb_degree = o.cheb_degree_phi;
    amg_build(P->amg_p, P->App, P->Bp, 1, app, P->stream);
    P->cur.amg_builds_phi += 1;
    if (!P->active_built) P->active_built = dalloc<uint8_t>(n);
    PFF_CUDA(cudaMemcpyAsync(P->active_built, P->active, n, cudaMemcpyDeviceToDevice, P->stream));
    P->amg_p_valid = true;
    P->phi_amg_age = 0;
  } else {
    AmgLevel& L0 = P->amg_p.lev[0];
    launch_stencil_dinv(m, n, 1, P->Kpp, L0.dinv, ap.mixed ? L0.dinvf : nullptr, P->stream);
    P->phi_amg_age += 1;
  }
  use_stencil(P->amg_p, P->Kpp, P->Kpp_f, 1);
}

// z = diag(V_u, V_phi) (S .* r) -- the right preconditioner of the scaled system
void precond_apply(pff_problem* P, const double* r, double* z) {
  const int64_t N = P->n_dofs, nu = (int64_t)P->dim * P->n_nodes;
  {
    ProfScope ps("vec_mul", 24.0 * N, P->stream);
    k_mul<<<grid_for(N, 256), 256, 0, P->stream>>>(N, P->op_S ? P->op_S : P->S, r, P->tmp);
  }
  PFF_LAUNCH("precond scale");
  if (P->overlap) {
    // the two diagonal blocks are independent: their V-cycles (whose coarse
    // levels are latency-bound) overlap on two streams
    if (!P->side) {
      PFF_CUDA(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
      PFF_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
      PFF_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    }
    PFF_CUDA(cudaEventRecord(P->ev_fork, P->stream));
    PFF_CUDA(cudaStreamWaitEvent(P->side, P->ev_fork, 0));
    amg_vcycle(P->amg_p, P->tmp + nu, z + nu, P->side);
    amg_vcycle(P->amg_u, P->tmp, z, P->stream);
    PFF_CUDA(cudaEventRecord(P->ev_join, P->side));
    PFF_CUDA(cudaStreamWaitEvent(P->stream, P->ev_join, 0));
  } else {
    amg_vcycle(P->amg_u, P->tmp, z, P->stream);
    amg_vcycle(P->amg_p, P->tmp + nu, z + nu, P->stream);
  }
}

__global__ void k_tri_rhs(int64_t n, const double* __restrict__ S, const double* __restrict__ y,
                          double* __restrict__ t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) t[i] -= S[i] * y[i];
}

// block lower-triangular form: z_u = V_u (S_u r_u), then
// z_phi = V_phi (S_phi (r_phi - [S^-1 G~ (z_u, 0)]_phi)) -- the exact coupling
// M_phi_u z_u of the reduced Jacobian, through the ordinary Jacobian apply
static void precond_apply_tri(pff_problem* P, const double* r, double* z) {
  const int64_t N = P->n_dofs, nu = (int64_t)P->dim * P->n_nodes, np = N - nu;
  const double* S = P->op_S ? P->op_S : P->S;
  if (!P->pc_tmp) P->pc_tmp = dalloc<double>(N);
  {
    ProfScope ps("vec_mul", 24.0 * N, P->stream);
    k_mul<<<grid_for(N, 256), 256, 0, P->stream>>>(N, S, r, P->tmp);
  }
  amg_vcycle(P->amg_u, P->tmp, z, P->stream);
  PFF_CUDA(cudaMemcpyAsync(P->pc_tmp, z, sizeof(double) * nu, cudaMemcpyDeviceToDevice, P->stream));
  PFF_CUDA(cudaMemsetAsync(P->pc_tmp + nu, 0, sizeof(double) * np, P->stream));
  apply_jacobian(P, P->apply_variant, P->pc_tmp, P->w, P->op_Sinv ? P->op_Sinv : P->Sinv);
  {
    ProfScope ps("vec_sub", 24.0 * np, P->stream);
    k_tri_rhs<<<grid_for(np, 256), 256, 0, P->stream>>>(np, S + nu, P->w + nu, P->tmp + nu);
  }
  amg_vcycle(P->amg_p, P->tmp + nu, z + nu, P->stream);
}

// The device work of one FGMRES iteration -- z = M v (preconditioner) and
// w = S^-1 G~ z (Jacobian apply) -- captured once as a CUDA graph on the fixed
// buffers g_in (v) and g_out (z), and recaptured whenever something it embeds
// changes (a hierarchy build, the scaling vectors, the apply variant, the
// precision or the stream overlap).  Small problems are launch-bound: the graph
// turns about 25 launches per iteration into one.  Returns false when the
// graph cannot be used (capture failed); the caller then launches directly.
constexpr int64_t ITER_GRAPH_MAX_DOFS = 1000000;

static bool iteration_graph(pff_problem* P) {
  const uint64_t key[8] = {P->amg_u.build_id, P->amg_p.build_id,
                           (uint64_t)(uintptr_t)(P->op_S ? P->op_S : P->S),
                           (uint64_t)(uintptr_t)(P->op_Sinv ? P->op_Sinv : P->Sinv),
                           (uint64_t)P->apply_variant, (uint64_t)P->precision,
                           (uint64_t)P->overlap, (uint64_t)(uintptr_t)P->stream};
  if (P->iter_graph && std::equal(key, key + 8, P->iter_key)) return true;
  if (P->iter_graph) {
    cudaGraphExecDestroy(P->iter_graph);
    P->iter_graph = nullptr;
  }
  const int64_t N = P->n_dofs;
  if (!P->g_in) P->g_in = dalloc<double>(N);
  if (!P->g_out) P->g_out = dalloc<double>(N);
  cudaStream_t s = P->stream;
  if (!s) return false;   // the legacy default stream cannot be captured
  if (P->overlap && !P->side) {
    PFF_CUDA(cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking));
    PFF_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
    PFF_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  }
  bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  cudaGraph_t g = nullptr;
  if (ok) {
    P->amg_u.inline_levels = P->amg_p.inline_levels = true;
    set_capturing(true);
    try {
      precond_apply(P, P->g_in, P->g_out);
      apply_jacobian(P, P->apply_variant, P->g_out, P->w, P->op_Sinv ? P->op_Sinv : P->Sinv);
    } catch (...) {
      ok = false;
    }
    set_capturing(false);
    P->amg_u.inline_levels = P->amg_p.inline_levels = false;
    if (cudaStreamEndCapture(s, &g) != cudaSuccess) ok = false;
  }
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
    P->iter_graph_kernels = kern;
    if (cudaGraphInstantiate(&P->iter_graph, g, 0) != cudaSuccess) {
      P->iter_graph = nullptr;
      ok = false;
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (!ok) return false;
  std::copy(key, key + 8, P->iter_key);
  return true;
}

static void precond(pff_problem* P, const pff_options& o, const double* r, double* z) {
  if (o.precond == PFF_PC_JACOBI) {
    PFF_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * P->n_dofs, cudaMemcpyDeviceToDevice, P->stream));
  } else if (o.precond == PFF_PC_AMG_TRI) {
    precond_apply_tri(P, r, z);   // uses P->w: free until the Jacobian apply that follows
  } else {
    precond_apply(P, r, z);
  }
}

// Restarted flexible GMRES (right preconditioned) for (S^-1 G~) x = b; b is
// already scaled.  Returns PFF_OK or PFF_ERR_NOT_CONVERGED.
// Orthogonalization: FP64 precision runs classical Gram-Schmidt twice (CGS2)
// in FP64.  Mixed precision runs one classical pass whose coefficients come
// from FP32 views of the vectors (the FP64 update keeps the Arnoldi relation
// exact), and a second pass only when the first cancelled most of w
// (||w_new|| < ||w|| / 8, the Daniel-Gragg-Kaufman-Stewart test); the basis is
// then orthonormal to about 1e-6, which leaves the residual estimate of the
// least-squares problem an upper bound to within that factor.
int fgmres(pff_problem* P, const pff_options& o, const double* b, double* x, int* iters) {
  const int m = std::min(60, std::max(2, o.krylov_restart));   // multidot partials hold 64 vectors
  ensure_krylov(P, m);
  const int64_t N = P->n_dofs;
  cudaStream_t s = P->stream;
  double* V = P->V;
  double* Z = P->Z;
  double* w = P->w;
  double* dh = P->h;            // [0, m+1): pass 1, [m+2, ...): pass 2, [2(m+2)]: ||w||^2
  double* hh = P->h_host;
  const unsigned g = grid_for(N, 256);
  // k_normalize is grid-stride and each block first forms the scale (an FP64
  // square root and divide, slow here): one resident wave of blocks
  const unsigned gn = std::min<unsigned>(g, (unsigned)sm_count() * 8u);
  const bool gs_mixed = P->precision == PFF_PREC_MIXED && m + 1 <= 64 &&
                        N <= (int64_t)GS_MAX_ROWS * GS_MAX_BLOCKS;
  const bool use_iter_graph = o.precond == PFF_PC_AMG && N <= ITER_GRAPH_MAX_DOFS && o.iter_graph != 0;
  // FP32 view of the basis for the projection coefficients of the mixed path
  if (gs_mixed && !P->Vf) P->Vf = dalloc<float>((size_t)(P->krylov_m + 1) * N);
  float* Vf = gs_mixed ? P->Vf : nullptr;
  PFF_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
  dot_dev(b, b, N, P->d_scalars, P->partials, s);
  const double beta0 = std::sqrt(fetch(P, P->d_scalars));
  *iters = 0;
  if (!(beta0 > 0.0)) return std::isfinite(beta0) ? PFF_OK : PFF_ERR_NAN;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  int total = 0;
  const double target = o.tol_linear * beta0;
  // r = b
  PFF_CUDA(cudaMemcpyAsync(w, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  double beta = beta0;
  while (true) {
    {
      ProfScope ps("normalize", (Vf ? 20.0 : 16.0) * N, s);
      k_normalize<<<gn, 256, 0, s>>>(N, w, P->d_scalars, V, Vf);   // d_scalars holds ||r||^2
    }
    PFF_LAUNCH("normalize");
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    double resid = beta;
    for (; j < m; ++j) {
      double* vj = V + (int64_t)j * N;
      double* zj = Z + (int64_t)j * N;
      if (use_iter_graph && iteration_graph(P)) {
        PFF_CUDA(cudaMemcpyAsync(P->g_in, vj, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        {
          ProfScope ps("iteration_graph", 0.0, s, P->iter_graph_kernels);
          PFF_CUDA(cudaGraphLaunch(P->iter_graph, s));
        }
        PFF_CUDA(cudaMemcpyAsync(zj, P->g_out, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      } else {
        precond(P, o, vj, zj);
        apply_jacobian(P, P->apply_variant, zj, w, P->op_Sinv ? P->op_Sinv : P->Sinv);
      }
      double hn = 0.0;
      if (gs_mixed) {
        // dh[0..j] = h, dh[j+1] = ||w||^2; dh[2(m+2)] = ||w - V h||^2
        gs_dot_dev(Vf, N, j + 1, w, N, P->gs_part, dh, s);
        gs_axpy_dev(V, N, j + 1, dh, w, N, P->gs_part, dh + 2 * (m + 2), s);
        PFF_CUDA(cudaMemcpyAsync(hh, dh, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, s));
        sync(P);
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i];
        if (hh[2 * (m + 2)] < hh[j + 1] / 64.0) {
          double* h2 = dh + (m + 2);
          gs_dot_dev(Vf, N, j + 1, w, N, P->gs_part, h2, s);
          gs_axpy_dev(V, N, j + 1, h2, w, N, P->gs_part, dh + 2 * (m + 2), s);
          PFF_CUDA(cudaMemcpyAsync(hh, dh, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, s));
          sync(P);
          for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] += hh[(m + 2) + i];
        }
        hn = std::sqrt(hh[2 * (m + 2)]);
      } else {
        // CGS2
        multidot_dev(V, N, j + 1, w, N, dh, P->partials, s);
        multi_axpy_dev(V, N, j + 1, dh, w, N, -1.0, s);
        multidot_dev(V, N, j + 1, w, N, dh + (m + 2), P->partials, s);
        multi_axpy_dev(V, N, j + 1, dh + (m + 2), w, N, -1.0, s);
        dot_dev(w, w, N, dh + 2 * (m + 2), P->partials, s);
        PFF_CUDA(cudaMemcpyAsync(hh, dh, sizeof(double) * 3 * (m + 2), cudaMemcpyDeviceToHost, s));
        sync(P);
        hn = std::sqrt(hh[2 * (m + 2)]);
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i] + hh[(m + 2) + i];
      }
      if (!std::isfinite(hn)) return PFF_ERR_NAN;
      H[(size_t)(j + 1) * m + j] = hn;
      // V_{j+1} = w / hn  (norm squared already on device)
      {
        ProfScope ps("normalize", (Vf ? 20.0 : 16.0) * N, s);
        k_normalize<<<gn, 256, 0, s>>>(N, w, dh + 2 * (m + 2), V + (int64_t)(j + 1) * N,
                                      Vf ? Vf + (int64_t)(j + 1) * N : nullptr);
      }
      PFF_LAUNCH("normalize");
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      const double r = std::hypot(a, bb);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? bb / r : 0.0;
      H[(size_t)j * m + j] = r;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      resid = std::fabs(gv[j + 1]);
      ++total;
      if (resid <= target || total >= o.max_krylov || hn == 0.0) {
        ++j;
        break;
      }
    }
    // y = H^-1 g, x += Z y
    for (int i = j - 1; i >= 0; --i) {
      double t = gv[i];
      for (int k = i + 1; k < j; ++k) t -= H[(size_t)i * m + k] * y[k];
      y[i] = H[(size_t)i * m + i] != 0.0 ? t / H[(size_t)i * m + i] : 0.0;
    }
    for (int i = 0; i < j; ++i) hh[i] = y[i];
    PFF_CUDA(cudaMemcpyAsync(dh, hh, sizeof(double) * j, cudaMemcpyHostToDevice, s));
    multi_axpy_dev(Z, N, j, dh, x, N, 1.0, s);
    *iters = total;
    if (resid <= target) {
      sync(P);
      return PFF_OK;
    }
    if (total >= o.max_krylov) {
      sync(P);
      return PFF_ERR_NOT_CONVERGED;
    }
    // explicit restart residual r = b - A x
    apply_jacobian(P, P->apply_variant, x, w, P->op_Sinv ? P->op_Sinv : P->Sinv);
    {
      ProfScope ps("vec_sub", 24.0 * N, s);
      k_sub<<<g, 256, 0, s>>>(N, b, w, w);
    }
    dot_dev(w, w, N, P->d_scalars, P->partials, s);
    beta = std::sqrt(fetch(P, P->d_scalars));
    if (beta <= target) return PFF_OK;
  }
}

void begin_loading_step(pff_problem* P, double p) {
  P->mat.p = p;
  launch_phi_tilde(P->mesh(), P->n_nodes, P->steps_done, P->phi_old, P->phi_prev, P->phit,
                   P->stream);
  P->uu_assembled = false;
  P->phi_assembled = false;
  P->amg_u_check = true;   // the displacement hierarchy may carry over (precond_setup decides)
  // M_uu and S depend on phi~ only
  launch_assemble_uu(P->mesh(), P->mat, P->n_nodes, P->phit, P->Kuu, P->stream);
  launch_scaling(P->mesh(), P->mat, P->n_nodes, P->Kuu, P->S, P->Sinv, P->stream);
  P->uu_assembled = true;
  P->in_step = true;
  P->F_ready = false;
  P->k = 0;
  P->have_prev = false;
  P->last_small = false;
  P->rho0 = 0.0;
  P->cur = pff_step_report{};
  sync(P);
}

static double scaled_norms(pff_problem* P, const double* F, double* l2) {
  launch_scaled_reduced(P->mesh(), P->n_nodes, F, P->Sinv, P->active, P->tmp, P->stream);
  nrm_inf_dev(P->tmp, P->n_dofs, P->d_scalars, P->partials, P->stream);
  dot_dev(P->tmp, P->tmp, P->n_dofs, P->d_scalars + 1, P->partials, P->stream);
  PFF_CUDA(cudaMemcpyAsync(P->h_scalars, P->d_scalars, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           P->stream));
  sync(P);
  if (l2) *l2 = std::sqrt(P->h_scalars[1]);
  return P->h_scalars[0];
}

// nodes whose active-set indicator is numerically zero (|indicator| <= tau)
static int count_ties(pff_problem* P, double tau) {
  const int64_t n = P->n_nodes;
  count_launch();
  PFF_CUDA(cudaMemsetAsync(P->counters + 2, 0, sizeof(int), P->stream));
  k_count_ties<<<grid_for(n, 256), 256, 0, P->stream>>>(n, P->indicator, tau, P->counters + 2);
  PFF_CUDA(cudaMemcpyAsync(P->h_counters + 2, P->counters + 2, sizeof(int), cudaMemcpyDeviceToHost,
                           P->stream));
  sync(P);
  return P->h_counters[2];
}

// inf-norm of the scaled reduced residual left in P->tmp by scaled_norms, without the tie rows
// (a node whose indicator is within the band meets complementarity as active and as free)
static double stop_norm(pff_problem* P, double band) {
  const int64_t n = P->n_nodes;
  count_launch();
  k_zero_ties<<<grid_for(n, 256), 256, 0, P->stream>>>(n, P->dim, P->indicator, band, P->tmp);
  PFF_LAUNCH("zero_ties");
  nrm_inf_dev(P->tmp, P->n_dofs, P->d_scalars, P->partials, P->stream);
  PFF_CUDA(cudaMemcpyAsync(P->h_scalars, P->d_scalars, sizeof(double), cudaMemcpyDeviceToHost,
                           P->stream));
  sync(P);
  return P->h_scalars[0];
}

int newton_iteration(pff_problem* P, const pff_options& o, pff_step_report* rep) {
  if (!P->in_step) fail(PFF_ERR_INVALID_ARG, "no loading step in progress (call pff_set_pressure)");
  cudaStream_t s = P->stream;
  const int64_t n = P->n_nodes;
  const int dim = P->dim;
  const int64_t N = P->n_dofs;
  pff_step_report& R = P->cur;
  // 1-2. residual and active set (the line search of the previous iteration may
  // already have evaluated it at the accepted state: same kernel, same inputs)
  if (!P->F_ready) compute_residual(P, P->u, P->phi, P->F);
  P->F_ready = false;
  compute_active_set(P, o.c, o.tol_active, o.tol_change, o.cycle_lock, P->have_prev);
  PFF_CUDA(cudaMemcpyAsync(P->h_counters, P->counters, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  double rho_l2 = 0.0;
  const double rho_inf = scaled_norms(P, P->F, &rho_l2);
  const int n_active = P->h_counters[0];
  const int n_changed = P->have_prev ? P->h_counters[1] : n_active;
  const int n_significant = P->have_prev ? P->h_counters[2] : n_active;
  if (!std::isfinite(rho_inf)) {
    R.status = PFF_ERR_NAN;
    if (rep) *rep = R;
    return PFF_ERR_NAN;
  }
  if (P->k == 0) R.rho0 = P->rho0 = rho_inf;
  R.rho = rho_inf;
  R.active = n_active;
  R.changed = n_changed;
  R.locked = P->h_counters[3];
  // 3. stopping test
  const double rho_tol = std::max(o.tol_newton * P->rho0, o.atol_newton);
  bool done = P->rho0 == 0.0;
  if (!done && P->have_prev && n_significant == 0 && P->last_small)
    done = rho_inf <= rho_tol || stop_norm(P, o.tol_change * P->mat.Gc / P->mat.eps) <= rho_tol;
  if (done) {
    R.converged = 1;
    R.newton_its = P->k;
    R.ties = count_ties(P, o.tol_active * P->mat.Gc / P->mat.eps);
    PFF_CUDA(cudaMemcpyAsync(P->h_counters, P->counters, sizeof(int), cudaMemcpyDeviceToHost, s));
    R.status = PFF_OK;
    if (rep) *rep = R;
    return PFF_OK;
  }
  if (P->k >= o.max_newton) {
    R.converged = 0;
    R.newton_its = P->k;
    R.status = PFF_ERR_NOT_CONVERGED;
    if (rep) *rep = R;
    return PFF_ERR_NOT_CONVERGED;
  }
  // 4. reduced Jacobian and right-hand side
  assemble_all(P);
  if (P->apply_auto) choose_apply(P);

  precond_setup(P, o, true);
  // 5. linear solve on the scaled system.  The displacement and phase-field
  // blocks of S^-1 F~ differ by orders of magnitude (displacements vs. a
  // dimensionless phase field), so each block's rows are further divided by the
  // norm of its own right-hand side: the FGMRES tolerance then applies to both
  // blocks instead of only the larger one.
  const int64_t nu = (int64_t)dim * n;
  scale_into(P->Sinv, P->Ft, P->tmp, N, s);
  dot_dev(P->tmp, P->tmp, nu, P->d_scalars + 4, P->partials, s);
  dot_dev(P->tmp + nu, P->tmp + nu, n, P->d_scalars + 5, P->partials, s);
  PFF_CUDA(cudaMemcpyAsync(P->h_scalars + 4, P->d_scalars + 4, 2 * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  sync(P);
  // a block already at round-off relative to the other is not amplified past 1e6
  const double bu0 = std::sqrt(P->h_scalars[4]), bp0 = std::sqrt(P->h_scalars[5]);
  const double floor_b = 1e-6 * std::sqrt(bu0 * bu0 + bp0 * bp0);
  const double bu = std::max(bu0, floor_b), bp = std::max(bp0, floor_b);
  const double wu = bu > 0.0 ? 1.0 / bu : 1.0, wp = bp > 0.0 ? 1.0 / bp : 1.0;
  launch_block_weights(s, N, nu, P->S, P->Sinv, wu, wp, P->Sw, P->Sinvw);
  scale_into(P->Sinvw, P->Ft, P->Ftrial, N, s);
  P->op_S = P->Sw;
  P->op_Sinv = P->Sinvw;
  int its = 0;
  // linear tolerance: fixed tol_linear, or (forcing_max > 0) the Eisenstat-Walker
  // forcing term eta_k = gamma (rho_k / rho_{k-1})^2 within [tol_linear, forcing_max],
  // eta_0 = forcing_max: early Newton steps need no accurate linear solve; the
  // Newton stopping test alone decides the accuracy of the converged solution
  pff_options ol = o;
  if (o.forcing_max > 0.0) {
    double eta = o.forcing_max;
    if (P->k > 0 && P->rho_last > 0.0) {
      const double q = rho_inf / P->rho_last;
      eta = std::min(o.forcing_max, 0.9 * q * q);
    }
    ol.tol_linear = std::max(o.tol_linear, eta);
  }
  P->rho_last = rho_inf;
  const int lrc = fgmres(P, ol, P->Ftrial, P->dU, &its);
  P->op_S = nullptr;
  P->op_Sinv = nullptr;
  R.krylov_its += its;
  R.krylov_its_max = std::max(R.krylov_its_max, its);
  if (lrc == PFF_ERR_NAN) {
    R.status = lrc;
    if (rep) *rep = R;
    return lrc;
  }
  {
    ProfScope ps("vec_add", 24.0 * N, s);
    k_add<<<grid_for(N, 256), 256, 0, s>>>(N, P->dUA, P->dU);
  }
  // step size test on the full step
  launch_update(s, n, dim, P->u, P->phi, P->phi_old, P->active, P->dU, 1.0, P->ut, P->phit_trial);
  nrm_inf_dev(P->dU, (int64_t)dim * n, P->d_scalars, P->partials, s);
  nrm_inf_dev(P->ut, (int64_t)dim * n, P->d_scalars + 1, P->partials, s);
  nrm_inf_dev(P->dU + (int64_t)dim * n, n, P->d_scalars + 2, P->partials, s);
  nrm_inf_dev(P->phit_trial, n, P->d_scalars + 3, P->partials, s);
  PFF_CUDA(cudaMemcpyAsync(P->h_scalars, P->d_scalars, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  sync(P);
  const double* hs = P->h_scalars;
  const bool small = hs[0] <= o.tol_step * hs[1] && hs[2] <= o.tol_step * hs[3];
  const double step_u = hs[1] > 0 ? hs[0] / hs[1] : hs[0];
  const double step_phi = hs[3] > 0 ? hs[2] / hs[3] : hs[2];
  // 6. line search
  double omega = 1.0;
  bool trial_is_next = false;   // Ftrial holds the residual at the accepted state
  if (!small) {
    for (int t = 0; t <= o.max_halvings; ++t) {
      if (t > 0)
        launch_update(s, n, dim, P->u, P->phi, P->phi_old, P->active, P->dU, omega, P->ut,
                      P->phit_trial);
      compute_residual(P, P->ut, P->phit_trial, P->Ftrial);
      double l2 = 0.0;
      scaled_norms(P, P->Ftrial, &l2);
      if (l2 < rho_l2) {
        trial_is_next = true;
        break;
      }
      if (t == o.max_halvings) {
        omega = 1.0;
        R.linesearch_fails += 1;
        launch_update(s, n, dim, P->u, P->phi, P->phi_old, P->active, P->dU, omega, P->ut,
                      P->phit_trial);
        break;
      }
      omega *= 0.5;
    }
  }
  if (verbose())
    std::fprintf(stderr,
                 "[pff] newton k=%d rho=%.3e rho0=%.3e active=%d changed=%d (outside band %d) krylov=%d "
                 "step_u=%.3e step_phi=%.3e small=%d omega=%g\n",
                 P->k, rho_inf, P->rho0, n_active, n_changed, n_significant, its, step_u, step_phi,
                 (int)small, omega);
  std::swap(P->u, P->ut);
  std::swap(P->phi, P->phit_trial);
  if (trial_is_next) {
    std::swap(P->F, P->Ftrial);
    P->F_ready = true;
  }
  P->last_small = small;
  P->have_prev = true;
  P->k += 1;
  R.newton_its = P->k;
  R.status = lrc;
  if (rep) *rep = R;
  sync(P);
  return PFF_OK;
}

void end_loading_step(pff_problem* P) {
  std::swap(P->phi_prev, P->phi_old);
  PFF_CUDA(cudaMemcpyAsync(P->phi_old, P->phi, sizeof(double) * P->n_nodes, cudaMemcpyDeviceToDevice,
                           P->stream));
  P->steps_done += 1;
  P->in_step = false;
  sync(P);
}

}  // namespace pff
