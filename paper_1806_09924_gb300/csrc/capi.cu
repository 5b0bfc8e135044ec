// extern "C" entry points of include/pff.h: argument checks, ownership of the
// device state, error translation.  All numerical work is in the kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <unordered_map>
#include <unordered_set>

#include "pff_internal.h"

namespace pff {

namespace {
thread_local std::string g_msg;
}

void set_error(int code, const std::string& msg) {
  (void)code;
  g_msg = msg;
}

void fail(int code, const std::string& msg) { throw Failure{code, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  cudaGetLastError();
  const int code = e == cudaErrorMemoryAllocation ? PFF_ERR_OOM : PFF_ERR_CUDA;
  throw Failure{code, std::string(what) + ": " + cudaGetErrorString(e)};
}

// Device memory.  While an AllocStream scope names a (non-default) stream, memory
// comes from the device's stream-ordered pool on that stream (cudaMallocAsync /
// cudaFreeAsync: no device-wide synchronization, freed blocks cached for reuse);
// otherwise plain cudaMalloc / cudaFree.
namespace {
thread_local cudaStream_t t_alloc_stream = nullptr;
std::mutex g_async_mu;
std::unordered_set<void*> g_async_ptrs;
std::unordered_map<void*, size_t> g_sizes;   // every live allocation and its size
int64_t g_bytes = 0, g_peak = 0;

void account(void* p, size_t bytes) {   // g_async_mu held
  g_sizes[p] = bytes;
  g_bytes += (int64_t)bytes;
  g_peak = std::max(g_peak, g_bytes);
}
bool g_pool_ready[64] = {false};

void prepare_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (g_pool_ready[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;   // keep freed blocks in this process's pool
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  g_pool_ready[dev] = true;
}
}  // namespace

AllocStream::AllocStream(cudaStream_t s) : prev_(t_alloc_stream) { t_alloc_stream = s; }
AllocStream::~AllocStream() { t_alloc_stream = prev_; }

void* dmalloc(size_t bytes) {
  void* p = nullptr;
  cudaError_t e;
  if (t_alloc_stream) {
    std::lock_guard<std::mutex> g(g_async_mu);
    prepare_pool();
    e = cudaMallocAsync(&p, bytes ? bytes : 16, t_alloc_stream);
    if (e == cudaSuccess) {
      g_async_ptrs.insert(p);
      account(p, bytes);
    }
  } else {
    e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e == cudaSuccess) {
      std::lock_guard<std::mutex> g(g_async_mu);
      account(p, bytes);
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Failure{PFF_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                   cudaGetErrorString(e)};
  }
  return p;
}

void dfree(void* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> g(g_async_mu);
    auto sz = g_sizes.find(p);
    if (sz != g_sizes.end()) {
      g_bytes -= (int64_t)sz->second;
      g_sizes.erase(sz);
    }
    auto it = g_async_ptrs.find(p);
    if (it != g_async_ptrs.end()) {
      g_async_ptrs.erase(it);
      // outside an AllocStream scope the owner has synchronized its stream first
      cudaFreeAsync(p, t_alloc_stream);
      return;
    }
  }
  cudaFree(p);
}

}  // namespace pff

using pff::fail;


namespace {

void need(bool ok, const char* msg) {
  if (!ok) fail(PFF_ERR_INVALID_ARG, msg);
}

void sync(pff_problem* P) { PFF_CUDA(cudaStreamSynchronize(P->stream)); }

void upload(pff_problem* P, double* dst, const double* src, size_t n) {
  PFF_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyHostToDevice, P->stream));
}

void refresh_phi_tilde(pff_problem* P) {
  pff::launch_phi_tilde(P->mesh(), P->n_nodes, P->steps_done, P->phi_old, P->phi_prev, P->phit,
                        P->stream);
  P->uu_assembled = false;
  P->phi_assembled = false;
  P->amg_u_valid = false;
  P->amg_p_valid = false;
  P->in_step = false;
  P->F_ready = false;
}

void release(pff_problem* P) {
  using pff::dfree;
  for (int a = 0; a < 3; ++a) dfree(P->X[a]);
  double* dbl[] = {P->u, P->phi, P->phi_old, P->phi_prev, P->phit, P->mass, P->S, P->Sinv,
                   P->Sw, P->Sinvw,
                   P->indicator, P->d_scalars, P->partials, P->Kuu, P->Kpu, P->Kpp, P->F,
                   P->Ft, P->dU, P->dUA, P->ut, P->phit_trial, P->Ftrial, P->Bu, P->Bp, P->xyz,
                   P->V, P->Z, P->w, P->h, P->tmp};
  for (double* p : dbl) dfree(p);
  dfree(P->Kuu_f);
  dfree(P->Kpp_f);
  dfree(P->gs_part);
  dfree(P->phit_built);
  dfree(P->active_built);
  dfree(P->pc_tmp);
  dfree(P->qp);
  dfree(P->Vf);
  if (P->side) {
    cudaStreamSynchronize(P->side);
    cudaStreamDestroy(P->side);
    P->side = nullptr;
  }
  if (P->iter_graph) cudaGraphExecDestroy(P->iter_graph);
  P->iter_graph = nullptr;
  dfree(P->g_in);
  dfree(P->g_out);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  P->ev_fork = P->ev_join = nullptr;
  dfree(P->active);
  dfree(P->active_prev);
  dfree(P->raw_prev);
  dfree(P->locked);
  dfree(P->toggles);
  dfree(P->counters);
  if (P->h_counters) cudaFreeHost(P->h_counters);
  if (P->h_scalars) cudaFreeHost(P->h_scalars);
  if (P->h_host) cudaFreeHost(P->h_host);
  P->Auu.release();
  P->App.release();
  P->amg_u.release();
  P->amg_p.release();
}

// crack rule of Section 4 (see pff_set_crack in include/pff.h)
std::vector<double> crack_field(const pff_problem* P, double l0) {
  const int d = P->dim;
  std::vector<double> phi((size_t)P->n_nodes, 1.0);
  const auto& X = P->hX;
  const int nx = P->nc[0], ny = P->nc[1], nz = d == 3 ? P->nc[2] : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        bool cut;
        if (d == 2) {
          cut = X[0][i] < l0 && X[0][i + 1] > -l0 && X[1][j] <= 0.0 && X[1][j + 1] >= 0.0;
        } else {
          const double px = std::min(std::max(0.0, X[0][i]), X[0][i + 1]);
          const double py = std::min(std::max(0.0, X[1][j]), X[1][j + 1]);
          cut = X[2][k] <= 0.0 && X[2][k + 1] >= 0.0 && px * px + py * py < l0 * l0;
        }
        if (!cut) continue;
        for (int c = 0; c < (1 << d); ++c) {
          const int64_t ii = i + (c & 1), jj = j + ((c >> 1) & 1), kk = k + ((c >> 2) & 1);
          phi[(size_t)(ii + P->nn[0] * (jj + (int64_t)P->nn[1] * kk))] = 0.0;
        }
      }
  return phi;
}

}  // namespace

namespace pff {

// cells of one axis whose closed interval contains x, with averaging weights
static std::vector<std::pair<int, double>> axis_columns(const std::vector<double>& X, double x) {
  std::vector<std::pair<int, double>> hits;
  const int n = (int)X.size() - 1;
  if (!(x >= X[0] && x <= X[n])) fail(PFF_ERR_INVALID_ARG, "COD point outside the domain");
  const int p = (int)(std::upper_bound(X.begin(), X.end(), x) - X.begin());
  for (int i = std::max(0, p - 2); i < std::min(n, p + 1); ++i)
    if (X[i] <= x && x <= X[i + 1]) hits.push_back({i, 0.0});
  for (auto& h : hits) h.second = 1.0 / hits.size();
  return hits;
}

std::vector<CodColumn> cod_columns(const pff_problem* P, int n_pts, const double* pts) {
  const int d = P->dim;
  std::vector<CodColumn> cols;
  cols.reserve((size_t)n_pts * (d == 3 ? 4 : 2));
  for (int k = 0; k < n_pts; ++k) {
    const double x = pts[k * (d - 1)];
    const auto cx = axis_columns(P->hX[0], x);
    std::vector<std::pair<int, double>> cy = {{0, 1.0}};
    if (d == 3) cy = axis_columns(P->hX[1], pts[k * 2 + 1]);
    for (auto& a : cx)
      for (auto& b : cy) {
        CodColumn c{};
        c.col[0] = a.first;
        c.xi[0] = (x - P->hX[0][a.first]) / (P->hX[0][a.first + 1] - P->hX[0][a.first]);
        if (d == 3) {
          const double y = pts[k * 2 + 1];
          c.col[1] = b.first;
          c.xi[1] = (y - P->hX[1][b.first]) / (P->hX[1][b.first + 1] - P->hX[1][b.first]);
        }
        c.w = a.second * b.second;
        c.point = k;
        cols.push_back(c);
      }
  }
  return cols;
}

}  // namespace pff

extern "C" void pff_default_options(pff_options* o);

namespace {
// defaults overridden by the caller's options, checked
pff_options resolve_options(const pff_options* opts) {
  pff_options o;
  pff_default_options(&o);
  if (opts) o = *opts;
  need(o.precision == PFF_PREC_FP64 || o.precision == PFF_PREC_MIXED, "unknown precision");
  need(o.krylov_restart >= 1 && o.max_krylov >= 1, "krylov_restart and max_krylov must be >= 1");
  need(o.cheb_degree >= 1, "cheb_degree must be >= 1");
  need(o.max_newton >= 0 && o.max_halvings >= 0, "negative iteration limit");
  need(o.tol_change >= 0.0 && o.tol_active >= 0.0, "negative active-set band");
  need(o.amg_reuse_tol >= 0.0, "negative amg_reuse_tol");
  need(o.forcing_max >= 0.0 && o.forcing_max < 1.0, "forcing_max must be in [0, 1)");
  need(o.amg_rebuild_phi >= 0.0 && o.amg_age_phi >= 1, "amg_rebuild_phi < 0 or amg_age_phi < 1");
  need(o.amg_levels_phi >= -1, "amg_levels_phi must be >= -1");
  need(o.cheb_degree_phi >= 0, "cheb_degree_phi must be >= 0");
  need(o.amg_rotations >= -1 && o.amg_rotations <= 1, "amg_rotations must be -1, 0 or 1");
  need(o.cheb_degree_coarse >= -1, "cheb_degree_coarse must be >= -1");
  need(o.precond == PFF_PC_AMG || o.precond == PFF_PC_JACOBI || o.precond == PFF_PC_AMG_TRI,
       "unknown precond");
  need(o.spmv_group == 0 || o.spmv_group == -1 || o.spmv_group == 1 || o.spmv_group == 2 ||
           o.spmv_group == 4 || o.spmv_group == 8 || o.spmv_group == 16 || o.spmv_group == 32 ||
           o.spmv_group == 64,
       "spmv_group must be 0, -1, 1, 2, 4, 8, 16, 32 or 64");
  return o;
}
}  // namespace

extern "C" {

void pff_default_options(pff_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = PFF_PREC_FP64;
  o->c = 0.1;
  o->tol_newton = 1e-10;
  o->tol_step = 1e-9;
  o->tol_linear = 1e-8;
  o->max_newton = 50;
  o->max_halvings = 10;
  o->cycle_lock = 3;
  o->krylov_restart = 40;
  o->max_krylov = 600;
  o->cheb_degree = 4;
  o->cheb_degree_coarse = -1;
  o->cheb_degree_phi = 4;
  o->amg_levels_phi = -1;
  o->amg_rotations = -1;
  o->amg_theta = 0.02;
  o->amg_coarse_max = 1000;
  o->apply_variant = PFF_APPLY_AUTO;
  o->precond = PFF_PC_AMG;
  o->cheb_ratio = 8.0;
  o->tol_active = 1e-10;
  o->atol_newton = 1e-14;
  o->tol_change = 1e-9;
  o->amg_reuse = 1;
  o->amg_reuse_tol = 0.05;
  o->precond_overlap = 1;
  o->iter_graph = 1;
  o->amg_rebuild_phi = 1e-3;
  o->amg_age_phi = 8;
}

int pff_check_options(const pff_options* opts) {
  API_BEGIN
  resolve_options(opts);
  API_END
}

const char* pff_last_error(void) { return pff::g_msg.c_str(); }

int pff_memory_usage(int64_t* current, int64_t* peak, int reset_peak) {
  std::lock_guard<std::mutex> g(pff::g_async_mu);
  if (current) *current = pff::g_bytes;
  if (peak) *peak = pff::g_peak;
  if (reset_peak) pff::g_peak = pff::g_bytes;
  return PFF_OK;
}

int pff_create_mesh(int dim, const int32_t* n_cells, const double* const* axis_coords,
                    pff_problem** out) {
  API_BEGIN
  need(out != nullptr, "out is NULL");
  *out = nullptr;
  *out = pff::create_problem(dim, n_cells, axis_coords, nullptr);
  API_END
}

}  // extern "C"

namespace pff {
// A problem whose set-up work and device memory are ordered on stream s (the
// stream-ordered pool when s is not the legacy default stream, so that
// creating and destroying problems does not synchronize the device while other
// problems solve); pff_create_mesh uses the legacy default stream.
pff_problem* create_problem(int dim, const int32_t* n_cells, const double* const* axis_coords,
                            cudaStream_t stream) {
  need(dim == 2 || dim == 3, "dim must be 2 or 3");
  need(n_cells && axis_coords, "n_cells / axis_coords is NULL");
  auto* P = new pff_problem();
  P->stream = stream;
  AllocStream alloc_scope(stream);
  try {
    P->dim = dim;
    int64_t nn = 1, nc = 1;
    for (int a = 0; a < dim; ++a) {
      need(n_cells[a] >= 1 && n_cells[a] < (1 << 24), "n_cells out of range");
      need(axis_coords[a] != nullptr, "axis coordinate array is NULL");
      P->nc[a] = n_cells[a];
      P->nn[a] = n_cells[a] + 1;
      P->hX[a].assign(axis_coords[a], axis_coords[a] + n_cells[a] + 1);
      for (int i = 0; i <= n_cells[a]; ++i)
        need(std::isfinite(P->hX[a][i]) && (i == 0 || P->hX[a][i] > P->hX[a][i - 1]),
             "axis coordinates must be finite and strictly increasing");
      nn *= P->nn[a];
      nc *= P->nc[a];
    }
    need(nn < (int64_t)1 << 31, "too many nodes");
    P->n_nodes = nn;
    P->n_cells = nc;
    P->n_dofs = (int64_t)(dim + 1) * nn;
    const int64_t n = nn, N = P->n_dofs;
    for (int a = 0; a < dim; ++a) {
      P->X[a] = pff::dalloc<double>(P->nn[a]);
      PFF_CUDA(cudaMemcpyAsync(P->X[a], P->hX[a].data(), sizeof(double) * P->nn[a],
                               cudaMemcpyHostToDevice, P->stream));
    }
    using pff::dalloc;
    P->u = dalloc<double>(n * dim);
    P->ut = dalloc<double>(n * dim);
    P->phi = dalloc<double>(n);
    P->phi_old = dalloc<double>(n);
    P->phi_prev = dalloc<double>(n);
    P->phit = dalloc<double>(n);
    P->phit_trial = dalloc<double>(n);
    P->mass = dalloc<double>(n);
    P->S = dalloc<double>(N);
    P->Sinv = dalloc<double>(N);
    P->Sw = dalloc<double>(N);
    P->Sinvw = dalloc<double>(N);
    P->indicator = dalloc<double>(n);
    P->active = dalloc<uint8_t>(n);
    P->active_prev = dalloc<uint8_t>(n);
    P->raw_prev = dalloc<uint8_t>(n);
    P->locked = dalloc<uint8_t>(n);
    P->toggles = dalloc<int>(n);
    P->counters = dalloc<int>(8);
    P->d_scalars = dalloc<double>(16);
    P->partials = dalloc<double>(65536);
    PFF_CUDA(cudaMallocHost(&P->h_counters, sizeof(int) * 8));
    PFF_CUDA(cudaMallocHost(&P->h_scalars, sizeof(double) * 16));
    const int NS = pff::n_slots(dim);
    P->Kuu = dalloc<double>((size_t)NS * dim * dim * n);
    P->Kpu = dalloc<double>((size_t)NS * dim * n);
    P->Kpp = dalloc<double>((size_t)NS * n);
    P->qp = dalloc<double>((size_t)pff::qp_doubles(dim, P->n_cells));
    P->F = dalloc<double>(N);
    P->Ft = dalloc<double>(N);
    P->dU = dalloc<double>(N);
    P->dUA = dalloc<double>(N);
    P->Ftrial = dalloc<double>(N);
    P->tmp = dalloc<double>(N);
    PFF_CUDA(cudaMemsetAsync(P->u, 0, sizeof(double) * n * dim, P->stream));
    PFF_CUDA(cudaMemsetAsync(P->active, 0, n, P->stream));
    PFF_CUDA(cudaMemsetAsync(P->raw_prev, 0, n, P->stream));
    PFF_CUDA(cudaMemsetAsync(P->locked, 0, n, P->stream));
    PFF_CUDA(cudaMemsetAsync(P->toggles, 0, sizeof(int) * n, P->stream));
    std::vector<double> ones((size_t)n, 1.0);
    PFF_CUDA(cudaMemcpyAsync(P->phi, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                             P->stream));
    PFF_CUDA(cudaMemcpyAsync(P->phi_old, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                             P->stream));
    PFF_CUDA(cudaMemcpyAsync(P->phi_prev, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                             P->stream));
    P->Bp = dalloc<double>(n);
    PFF_CUDA(cudaMemcpyAsync(P->Bp, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                             P->stream));
    const auto m = P->mesh();
    pff::launch_lumped_mass(m, n, P->mass, P->stream);
    P->Bu = dalloc<double>((size_t)n * dim * (dim == 2 ? 3 : 6));
    pff::launch_rigid_modes(m, n, P->Bu, P->stream);
    P->xyz = dalloc<double>((size_t)n * dim);
    pff::launch_node_coords(m, n, P->xyz, P->stream);
    pff::build_stencil_bsr_structure(m, n, dim, P->Auu, P->stream);
    pff::build_stencil_bsr_structure(m, n, 1, P->App, P->stream);
    const double E = 1.0, nu = 0.2;
    P->mat.mu = E / (2.0 * (1.0 + nu));
    P->mat.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    refresh_phi_tilde(P);
    sync(P);
  } catch (...) {
    cudaStreamSynchronize(P->stream);
    release(P);
    delete P;
    throw;
  }
  return P;
}
}  // namespace pff

extern "C" {

int pff_set_material(pff_problem* P, double E, double nu, double Gc, double kappa, double eps) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  need(E > 0 && std::isfinite(E), "E must be > 0");
  need(nu >= 0 && nu < 0.5, "nu must be in [0, 0.5)");
  need(Gc > 0 && std::isfinite(Gc), "Gc must be > 0");
  need(kappa >= 0 && kappa < 1, "kappa must be in [0, 1)");
  need(eps > 0 && std::isfinite(eps), "eps must be > 0");
  P->mat.E = E;
  P->mat.nu = nu;
  P->mat.Gc = Gc;
  P->mat.kappa = kappa;
  P->mat.eps = eps;
  P->mat.mu = E / (2.0 * (1.0 + nu));
  P->mat.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  P->uu_assembled = false;
  P->phi_assembled = false;
  P->amg_u_valid = false;
  P->amg_p_valid = false;
  P->in_step = false;
  P->F_ready = false;
  API_END
}

int pff_set_pressure(pff_problem* P, double p) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  need(std::isfinite(p), "pressure must be finite");
  pff::begin_loading_step(P, p);
  API_END
}

int pff_set_crack(pff_problem* P, double l0) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  need(l0 > 0 && std::isfinite(l0), "l0 must be > 0");
  const auto phi = crack_field(P, l0);
  const size_t n = (size_t)P->n_nodes;
  upload(P, P->phi, phi.data(), n);
  upload(P, P->phi_old, phi.data(), n);
  upload(P, P->phi_prev, phi.data(), n);
  PFF_CUDA(cudaMemsetAsync(P->u, 0, sizeof(double) * n * P->dim, P->stream));
  P->steps_done = 0;
  refresh_phi_tilde(P);
  sync(P);
  API_END
}

int pff_set_state(pff_problem* P, const double* u, const double* phi, const double* phi_old,
                  const double* phi_prev, int steps_done) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  need(steps_done >= 0, "steps_done must be >= 0");
  const size_t n = (size_t)P->n_nodes;
  if (u) upload(P, P->u, u, n * P->dim);
  if (phi) upload(P, P->phi, phi, n);
  if (phi_old) upload(P, P->phi_old, phi_old, n);
  if (phi_prev) upload(P, P->phi_prev, phi_prev, n);
  P->steps_done = steps_done;
  refresh_phi_tilde(P);
  sync(P);
  API_END
}

int pff_set_state_dev(pff_problem* P, const double* u, const double* phi, const double* phi_old,
                      const double* phi_prev, int steps_done) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  need(steps_done >= 0, "steps_done must be >= 0");
  const size_t n = (size_t)P->n_nodes;
  const auto d2d = cudaMemcpyDeviceToDevice;
  if (u) PFF_CUDA(cudaMemcpyAsync(P->u, u, sizeof(double) * n * P->dim, d2d, P->stream));
  if (phi) PFF_CUDA(cudaMemcpyAsync(P->phi, phi, sizeof(double) * n, d2d, P->stream));
  if (phi_old) PFF_CUDA(cudaMemcpyAsync(P->phi_old, phi_old, sizeof(double) * n, d2d, P->stream));
  if (phi_prev) PFF_CUDA(cudaMemcpyAsync(P->phi_prev, phi_prev, sizeof(double) * n, d2d, P->stream));
  P->steps_done = steps_done;
  refresh_phi_tilde(P);
  API_END
}

int pff_newton_step(pff_problem* P, const pff_options* opts, pff_step_report* rep) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  pff::AllocStream alloc_scope(P->stream);
  const pff_options o = resolve_options(opts);
  if (o.apply_variant == PFF_APPLY_MATFREE || o.apply_variant == PFF_APPLY_ASSEMBLED)
    P->apply_variant = o.apply_variant;
  P->apply_auto = o.apply_variant == PFF_APPLY_AUTO;
  const int rc = pff::newton_iteration(P, o, rep);
  if (rc != PFF_OK) {
    pff::set_error(rc, "Newton iteration failed");
    return rc;
  }
  API_END
}

int pff_end_loading_step(pff_problem* P) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  pff::end_loading_step(P);
  API_END
}

int pff_solve_loading_steps(pff_problem* P, int n_steps, const double* p_schedule,
                            const pff_options* opts, pff_step_report* reports) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  pff::AllocStream alloc_scope(P->stream);
  need(n_steps >= 0 && (n_steps == 0 || p_schedule != nullptr), "bad schedule");
  const pff_options o = resolve_options(opts);
  if (o.apply_variant == PFF_APPLY_MATFREE || o.apply_variant == PFF_APPLY_ASSEMBLED)
    P->apply_variant = o.apply_variant;
  P->apply_auto = o.apply_variant == PFF_APPLY_AUTO;
  int rc_all = PFF_OK;
  for (int st = 0; st < n_steps; ++st) {
    const auto t0 = std::chrono::steady_clock::now();
    pff::begin_loading_step(P, p_schedule[st]);
    pff_step_report r{};
    int rc = PFF_OK;
    while (true) {
      rc = pff::newton_iteration(P, o, &r);
      if (rc != PFF_OK || r.converged) break;
    }
    pff::end_loading_step(P);
    r.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    r.status = rc;
    if (reports) reports[st] = r;
    if (rc != PFF_OK) {
      rc_all = rc;
      pff::set_error(rc, "loading step " + std::to_string(st) + " failed");
      return rc_all;
    }
  }
  API_END
}

int pff_eval_tcv_cod(pff_problem* P, int n_pts, const double* pts, double* tcv, double* cod) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  pff::AllocStream alloc_scope(P->stream);
  need(n_pts >= 0 && (n_pts == 0 || pts != nullptr), "bad COD points");
  const auto m = P->mesh();
  if (tcv) {
    pff::tcv_dev(m, P->n_cells, P->u, P->phi, P->d_scalars, P->partials, P->stream);
    PFF_CUDA(cudaMemcpyAsync(P->h_scalars, P->d_scalars, sizeof(double), cudaMemcpyDeviceToHost,
                             P->stream));
    sync(P);
    *tcv = P->h_scalars[0];
  }
  if (cod && n_pts > 0) {
    const std::vector<pff::CodColumn> cols = pff::cod_columns(P, n_pts, pts);
    const int nc = (int)cols.size();
    auto* dcols = pff::dalloc<pff::CodColumn>(nc);
    double* dout = pff::dalloc<double>(nc);
    PFF_CUDA(cudaMemcpyAsync(dcols, cols.data(), sizeof(pff::CodColumn) * nc, cudaMemcpyHostToDevice,
                             P->stream));
    pff::cod_dev(m, dcols, nc, P->u, P->phi, dout, n_pts, P->stream);
    std::vector<double> hout(nc);
    PFF_CUDA(cudaMemcpyAsync(hout.data(), dout, sizeof(double) * nc, cudaMemcpyDeviceToHost, P->stream));
    sync(P);
    pff::dfree(dcols);
    pff::dfree(dout);
    for (int k = 0; k < n_pts; ++k) cod[k] = 0.0;
    for (int c = 0; c < nc; ++c) cod[cols[c].point] += hout[c];
  }
  API_END
}

int pff_cell_indicators_dev(pff_problem* P, double* eta2_dev) {
  API_BEGIN
  need(P != nullptr && eta2_dev != nullptr, "NULL argument");
  pff::jump_indicator_dev(P->mesh(), P->n_cells, P->u, eta2_dev, P->stream);
  API_END
}

}  // extern "C"

namespace {
// Marking and splitting of one axis (Section 3 refinement strategy, tensor-product
// form): interval i is split when its slab sum S[i] is positive and reaches theta
// times the axis maximum, or when the slab reaches the crack region
// (minphi[i] < phi_band) while the interval is longer than h_band; a split adds
// the midpoint when it lies strictly inside.  out holds up to 2 nc + 1 values;
// returns the new cell count.
int mark_axis(int nc, const double* x, const double* S, const double* minphi, double theta,
              double h_band, double phi_band, double* out) {
  double smax = 0.0;
  for (int i = 0; i < nc; ++i) smax = std::max(smax, S[i]);
  int k = 0;
  for (int i = 0; i < nc; ++i) {
    out[k++] = x[i];
    const bool by_eta = smax > 0.0 && S[i] > 0.0 && S[i] >= theta * smax;
    const bool by_band = minphi[i] < phi_band && x[i + 1] - x[i] > h_band;
    const double mid = 0.5 * (x[i] + x[i + 1]);
    if ((by_eta || by_band) && mid > x[i] && mid < x[i + 1]) out[k++] = mid;
  }
  out[k++] = x[nc];
  return k - 1;
}

void check_refine_args(double theta, double h_band, double phi_band) {
  need(theta >= 0 && std::isfinite(theta), "theta must be finite and >= 0");
  need(h_band >= 0 && std::isfinite(h_band), "h_band must be finite and >= 0");
  need(std::isfinite(phi_band), "phi_band must be finite");
}
}  // namespace

extern "C" {

int pff_mark_axes(int dim, const int32_t* n_cells, const double* const* coords,
                  const double* const* slab_eta2, const double* const* slab_minphi, double theta,
                  double h_band, double phi_band, int32_t* n_cells_out, double* const* coords_out) {
  API_BEGIN
  need(dim == 2 || dim == 3, "dim must be 2 or 3");
  need(n_cells && coords && slab_eta2 && slab_minphi && n_cells_out && coords_out, "NULL argument");
  check_refine_args(theta, h_band, phi_band);
  for (int a = 0; a < dim; ++a) {
    need(n_cells[a] >= 1, "n_cells must be >= 1");
    need(coords[a] && slab_eta2[a] && slab_minphi[a] && coords_out[a], "NULL axis array");
    for (int i = 0; i < n_cells[a]; ++i)
      need(coords[a][i + 1] > coords[a][i], "axis coordinates must be strictly increasing");
  }
  for (int a = 0; a < dim; ++a)
    n_cells_out[a] = mark_axis(n_cells[a], coords[a], slab_eta2[a], slab_minphi[a], theta, h_band,
                               phi_band, coords_out[a]);
  API_END
}

int pff_refine_axes(pff_problem* P, double theta, double h_band, double phi_band,
                    int32_t* n_cells_out, double* const* coords_out) {
  API_BEGIN
  need(P != nullptr && n_cells_out != nullptr && coords_out != nullptr, "NULL argument");
  check_refine_args(theta, h_band, phi_band);
  for (int a = 0; a < P->dim; ++a) need(coords_out[a] != nullptr, "coords_out[a] is NULL");
  pff::AllocStream alloc_scope(P->stream);
  const auto m = P->mesh();
  int slabs = 0;
  for (int a = 0; a < P->dim; ++a) slabs += P->nc[a];
  double* eta2 = pff::dalloc<double>(P->n_cells);
  double* red = pff::dalloc<double>(2 * (size_t)slabs);
  pff::jump_indicator_dev(m, P->n_cells, P->u, eta2, P->stream);
  pff::slab_reduce_dev(m, eta2, P->phi, red, red + slabs, P->stream);
  std::vector<double> h(2 * (size_t)slabs);
  PFF_CUDA(cudaMemcpyAsync(h.data(), red, sizeof(double) * 2 * slabs, cudaMemcpyDeviceToHost,
                           P->stream));
  sync(P);
  pff::dfree(eta2);
  pff::dfree(red);
  int off = 0;
  for (int a = 0; a < P->dim; ++a) {
    n_cells_out[a] = mark_axis(P->nc[a], P->hX[a].data(), h.data() + off, h.data() + slabs + off,
                               theta, h_band, phi_band, coords_out[a]);
    off += P->nc[a];
  }
  API_END
}

int pff_transfer_state(pff_problem* src, pff_problem* dst, int fields) {
  API_BEGIN
  need(src != nullptr && dst != nullptr, "problem is NULL");
  need(src != dst, "src and dst must be different problems");
  need(src->dim == dst->dim, "src and dst differ in dimension");
  need((fields & ~(PFF_FIELD_U | PFF_FIELD_PHI | PFF_FIELD_PHI_OLD | PFF_FIELD_PHI_PREV)) == 0,
       "unknown field flag");
  const int dim = src->dim;
  for (int a = 0; a < dim; ++a)
    need(dst->hX[a].front() >= src->hX[a].front() && dst->hX[a].back() <= src->hX[a].back(),
         "dst mesh leaves the src mesh's box");
  // per axis: source interval (last one whose left end is <= the new coordinate)
  // and local coordinate of every new axis coordinate
  std::vector<int> hc[3];
  std::vector<double> ht[3];
  for (int a = 0; a < dim; ++a) {
    const std::vector<double>& x = src->hX[a];
    const int n = (int)x.size() - 1;
    for (double xn : dst->hX[a]) {
      int i = (int)(std::upper_bound(x.begin(), x.end(), xn) - x.begin()) - 1;
      i = std::min(std::max(i, 0), n - 1);
      hc[a].push_back(i);
      ht[a].push_back((xn - x[i]) / (x[i + 1] - x[i]));
    }
  }
  sync(src);
  pff::AllocStream alloc_scope(dst->stream);
  const int* dc[3] = {nullptr, nullptr, nullptr};
  const double* dt[3] = {nullptr, nullptr, nullptr};
  std::vector<void*> temps;
  for (int a = 0; a < dim; ++a) {
    int* c = pff::dalloc<int>(hc[a].size());
    double* t = pff::dalloc<double>(ht[a].size());
    PFF_CUDA(cudaMemcpyAsync(c, hc[a].data(), sizeof(int) * hc[a].size(), cudaMemcpyHostToDevice,
                             dst->stream));
    PFF_CUDA(cudaMemcpyAsync(t, ht[a].data(), sizeof(double) * ht[a].size(), cudaMemcpyHostToDevice,
                             dst->stream));
    dc[a] = c;
    dt[a] = t;
    temps.push_back(c);
    temps.push_back(t);
  }
  struct Field {
    int flag;
    const double* s;
    double* d;
    int ncomp;
  } list[] = {{PFF_FIELD_U, src->u, dst->u, dim},
              {PFF_FIELD_PHI, src->phi, dst->phi, 1},
              {PFF_FIELD_PHI_OLD, src->phi_old, dst->phi_old, 1},
              {PFF_FIELD_PHI_PREV, src->phi_prev, dst->phi_prev, 1}};
  for (const Field& f : list)
    if (fields & f.flag)
      pff::transfer_dev(dim, dst->nn, src->nn, dc, dt, f.s, f.ncomp, f.d, dst->stream);
  sync(dst);
  for (void* p : temps) pff::dfree(p);
  if (fields & PFF_FIELD_PHI_OLD) dst->steps_done = src->steps_done;
  refresh_phi_tilde(dst);
  sync(dst);
  API_END
}

int pff_get_solution(pff_problem* P, double* u, double* phi, uint8_t* active) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  const size_t n = (size_t)P->n_nodes;
  if (u) PFF_CUDA(cudaMemcpyAsync(u, P->u, sizeof(double) * n * P->dim, cudaMemcpyDeviceToHost, P->stream));
  if (phi) PFF_CUDA(cudaMemcpyAsync(phi, P->phi, sizeof(double) * n, cudaMemcpyDeviceToHost, P->stream));
  if (active) PFF_CUDA(cudaMemcpyAsync(active, P->active, n, cudaMemcpyDeviceToHost, P->stream));
  sync(P);
  API_END
}

int pff_set_stream(pff_problem* P, void* stream) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  sync(P);
  P->stream = static_cast<cudaStream_t>(stream);
  API_END
}

int pff_get_sizes(const pff_problem* P, int* dim, int64_t* n_nodes, int64_t* n_dofs) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  if (dim) *dim = P->dim;
  if (n_nodes) *n_nodes = P->n_nodes;
  if (n_dofs) *n_dofs = P->n_dofs;
  API_END
}

void pff_destroy(pff_problem* P) {
  if (!P) return;
  cudaStreamSynchronize(P->stream);
  {
    pff::AllocStream alloc_scope(P->stream);   // pool memory goes back on the problem's stream
    release(P);
  }
  cudaStreamSynchronize(P->stream);
  delete P;
}

int pff_residual_dev(pff_problem* P, double* F_dev) {
  API_BEGIN
  need(P != nullptr && F_dev != nullptr, "NULL argument");
  pff::compute_residual(P, P->u, P->phi, F_dev);
  API_END
}

int pff_active_set_dev(pff_problem* P, double c, uint8_t* active_dev, double* indicator_dev) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  need(c > 0 && std::isfinite(c), "c must be > 0");
  pff::compute_residual(P, P->u, P->phi, P->F);
  pff::compute_active_set(P, c, 1e-10, 1e-9, 1 << 30, false);
  if (active_dev)
    PFF_CUDA(cudaMemcpyAsync(active_dev, P->active, P->n_nodes, cudaMemcpyDeviceToDevice, P->stream));
  if (indicator_dev)
    PFF_CUDA(cudaMemcpyAsync(indicator_dev, P->indicator, sizeof(double) * P->n_nodes,
                             cudaMemcpyDeviceToDevice, P->stream));
  P->phi_assembled = false;
  API_END
}

int pff_assemble(pff_problem* P) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  pff::compute_residual(P, P->u, P->phi, P->F);
  pff::assemble_all(P);
  API_END
}

int pff_apply_jacobian_dev(pff_problem* P, int variant, const double* x_dev, double* y_dev) {
  API_BEGIN
  need(P != nullptr && x_dev && y_dev, "NULL argument");
  need(variant == PFF_APPLY_ASSEMBLED || variant == PFF_APPLY_MATFREE, "bad variant");
  pff::apply_jacobian(P, variant, x_dev, y_dev, nullptr);
  API_END
}

int pff_precond_setup(pff_problem* P, const pff_options* opts) {
  API_BEGIN
  need(P != nullptr, "problem is NULL");
  pff::AllocStream alloc_scope(P->stream);
  need(P->phi_assembled, "call pff_assemble first");
  const pff_options o = resolve_options(opts);
  P->amg_u_valid = false;
  P->amg_p_valid = false;
  pff::precond_setup(P, o);
  sync(P);
  API_END
}

int pff_precond_apply_dev(pff_problem* P, const double* r_dev, double* z_dev) {
  API_BEGIN
  need(P != nullptr && r_dev && z_dev, "NULL argument");
  need(P->amg_u.built && P->amg_p.built, "call pff_precond_setup first");
  const int64_t nu = (int64_t)P->dim * P->n_nodes;
  pff::amg_vcycle(P->amg_u, r_dev, z_dev, P->stream);
  pff::amg_vcycle(P->amg_p, r_dev + nu, z_dev + nu, P->stream);
  API_END
}

int pff_linear_solve_dev(pff_problem* P, const pff_options* opts, const double* b_dev,
                         double* x_dev, int* iters) {
  API_BEGIN
  need(P != nullptr && b_dev && x_dev, "NULL argument");
  pff::AllocStream alloc_scope(P->stream);
  need(P->phi_assembled, "call pff_assemble first");
  const pff_options o = resolve_options(opts);
  if (o.precond != PFF_PC_JACOBI)
    need(P->amg_u.built && P->amg_p.built, "call pff_precond_setup first");
  if (o.apply_variant == PFF_APPLY_MATFREE || o.apply_variant == PFF_APPLY_ASSEMBLED)
    P->apply_variant = o.apply_variant;
  P->apply_auto = o.apply_variant == PFF_APPLY_AUTO;
  const int64_t N = P->n_dofs;
  pff::ensure_krylov(P, std::max(2, o.krylov_restart));
  // scaled right-hand side Sinv .* b into scratch, solution into x
  double* bs = P->Ftrial;
  pff::scale_into(P->Sinv, b_dev, bs, N, P->stream);
  int its = 0;
  const int rc = pff::fgmres(P, o, bs, x_dev, &its);
  if (iters) *iters = its;
  sync(P);
  if (rc != PFF_OK) {
    pff::set_error(rc, "FGMRES did not converge");
    return rc;
  }
  API_END
}

}  // extern "C"
