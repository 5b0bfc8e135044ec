// Internal declarations of the GB300 phase-field fracture library.
//
// Layers (bottom to top):
//   fe_kernels.cu  -- Q1 element-batched kernels: residual of Formulation 1,
//                     stencil assembly of the Section 3.1 Jacobian blocks,
//                     matrix-free and assembled Jacobian applies, active set,
//                     phi~ extrapolation, lumped mass, scaling, TCV / COD.
//   linalg.cu      -- deterministic reductions, scans, vector kernels, BSR SpMV,
//                     Chebyshev smoothing, dense coarse solve.
//   amg.cu         -- smoothed-aggregation AMG hierarchy built on the device
//                     and the V-cycle.
//   solver.cu      -- FGMRES with the block-diagonal preconditioner and the
//                     semi-smooth Newton / primal-dual active-set driver.
//   capi.cu        -- the extern "C" entry points of include/pff.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/pff.h"

namespace pff {

// ------------------------------------------------------------------ errors --
struct Error {
  int code;
  std::string msg;
};

// exception carrying a PFF_ERR_* code to the extern "C" boundary
struct Failure {
  int code;
  std::string msg;
};

void set_error(int code, const std::string& msg);
[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define PFF_CUDA(x) ::pff::check_cuda((x), #x)
#define PFF_LAUNCH(what) ::pff::check_cuda(cudaGetLastError(), what)

// Body of an extern "C" entry point: a Failure returns its code, a failed host
// allocation PFF_ERR_OOM, any other exception PFF_ERR_INVALID_ARG; the message
// is kept for pff_last_error.
#define API_BEGIN try {
#define API_END                                            \
  }                                                        \
  catch (const ::pff::Failure& f) {                        \
    ::pff::set_error(f.code, f.msg);                       \
    return f.code;                                         \
  }                                                        \
  catch (const std::bad_alloc&) {                          \
    ::pff::set_error(PFF_ERR_OOM, "host allocation failed"); \
    return PFF_ERR_OOM;                                    \
  }                                                        \
  catch (const std::exception& e) {                        \
    ::pff::set_error(PFF_ERR_INVALID_ARG, e.what());       \
    return PFF_ERR_INVALID_ARG;                            \
  }                                                        \
  return PFF_OK;

// ------------------------------------------------------- launch accounting --
// Every kernel launch is counted; when profiling is enabled, the launches of a
// ProfScope are also timed with a CUDA event pair and credited with their
// algorithmic bytes (each input / output array moved once).
void count_launch(int k = 1);
// while a stream is being captured into a graph, launches are neither counted
// nor timed (the graph's replays are); their algorithmic bytes are summed, and
// captured_bytes() returns the sum since capture started (the bytes of one replay)
void set_capturing(bool on);
double captured_bytes();
// diagnostics on stderr when the environment variable PFF_VERBOSE is set
bool verbose();
// Autotuner choices kept in the file named by PFF_TUNE_CACHE (when set): a choice
// found there is reused without timing, every new choice is written there.
bool tune_lookup(const std::string& key, int* value);
void tune_store(const std::string& key, int value);
class ProfScope {
 public:
  ProfScope(const char* name, double bytes, cudaStream_t s, int kernels = 1);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* name_;
  double bytes_;
  cudaStream_t s_;
  void* a_;
};

// ------------------------------------------------------------ device memory --
void* dmalloc(size_t bytes);
void dfree(void* p);
// Scope in which dmalloc / dfree are stream-ordered on stream s (a non-default
// stream; with s == nullptr the plain synchronous calls are used).
class AllocStream {
 public:
  explicit AllocStream(cudaStream_t s);
  ~AllocStream();

 private:
  cudaStream_t prev_;
};
template <class T>
T* dalloc(size_t n) {
  return static_cast<T*>(dmalloc(n * sizeof(T) + 16));
}

#ifdef __CUDACC__
// FP32 view of a double from its high word: sign, exponent re-biased, 20 mantissa
// bits (truncated; relative error < 2^-20), integer operations only.
// |x| < 2^-126 gives 0, |x| >= 2^128 gives inf.
__device__ __forceinline__ float f32_view(double x) {
  const unsigned hw = (unsigned)__double2hiint(x);
  const unsigned a = hw & 0x7fffffffu;
  unsigned f = a >= (1151u << 20) ? 0x7f800000u : ((a - (896u << 20)) << 3);
  f = a >= (897u << 20) ? f : 0u;
  return __uint_as_float(f | (hw & 0x80000000u));
}
#endif

// grid size for n threads of block b, capped
inline unsigned grid_for(int64_t n, int block, int64_t cap = 1 << 30) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// ------------------------------------------------------------------- mesh ---
struct MeshDev {
  int dim;
  int nn[3];      // nodes per axis
  int nc[3];      // cells per axis
  const double* X[3];  // device axis coordinates
};

// ------------------------------------------------------------ BSR matrices --
struct Bsr {
  int nrows = 0, ncols = 0;   // block rows / cols
  int br = 1, bc = 1;         // block size
  int64_t nnzb = 0;
  int* rowptr = nullptr;      // nrows + 1
  int* col = nullptr;         // nnzb, sorted within a row
  double* val = nullptr;      // nnzb * br * bc, block row-major
  float* valf = nullptr;      // FP32 copy (mixed precision)
  int group = 0;              // lanes per block row of the vector kernels: 0 = by row length,
                              // 1..32 = fixed, -1 = one thread per scalar row (reference),
                              // BSR_SELL = the sliced copy below (FP32 values)
  // SELL-32 copy: slices of 32 block rows; slice s holds sell_off[s+1] - sell_off[s]
  // entry columns of 32 blocks (its longest row); block k of row 32 s + l sits at entry
  // (sell_off[s] + k) * 32 + l, its element e at value (((sell_off[s] + k) * bb + e) * 32 + l)
  int* sell_off = nullptr;
  int* sell_col = nullptr;
  float* sell_valf = nullptr;
  void release();
};

// ------------------------------------------------------------------- AMG ---
struct AmgLevel {
  Bsr A, P, R;
  double* dinv = nullptr;     // inverse scalar diagonal (n scalar rows)
  float* dinvf = nullptr;
  double lmax = 1.0;          // estimate of the largest eigenvalue of D^-1 A
  int n = 0;                  // scalar rows
  bool terminal = false;      // no coarser level (every row isolated): smoothing only
  // the finest level may smooth on the assembled node stencil (slot-major,
  // block size A.br) instead of its BSR copy
  bool stencil = false;
  MeshDev mesh{};
  const double* st = nullptr;
  const float* stf = nullptr;
  bool stf_node_major = false;  // stf in the node-major 2d displacement layout
  // V-cycle work vectors (stored as doubles; FP32 cycles reinterpret them)
  double *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *t = nullptr;
};

struct Amg {
  std::vector<AmgLevel> lev;
  int nc = 0;                 // coarsest size (scalar)
  double* cinv = nullptr;     // dense inverse of the coarsest operator (nc x nc)
  float* cinvf = nullptr;
  double *cx = nullptr, *cb = nullptr;
  bool mixed = false;
  int cheb_degree = 2;
  int cheb_degree_coarse = 2;  // levels >= 1
  double cheb_ratio = 30.0;
  int built = 0;
  uint64_t build_id = 0;      // distinct for every build (process-wide counter)
  // levels 1.. captured as one CUDA graph (see coarse_cycle in amg.cu)
  bool use_graph = true;
  bool inline_levels = false; // run levels 1.. as ordinary launches (inside an outer capture)
  cudaGraphExec_t graph = nullptr;
  int graph_kernels = 0;
  double graph_bytes = 0.0;   // algorithmic bytes of one replay (sum over its kernels)
  cudaStream_t cap_stream = nullptr;
  void release();
};

struct AmgParams {
  double theta = 0.08;
  int coarse_max = 320;
  int cheb_degree = 2;
  int cheb_degree_coarse = 2;
  double cheb_ratio = 30.0;
  bool mixed = false;
  int max_levels = 20;
  // fine-level node coordinates (n x coord_dim, device); when given, strength
  // is measured on the distance Laplacian (theta) with a matrix drop (mdrop)
  const double* coords = nullptr;
  int coord_dim = 0;
  double mdrop = 1e-3;
  bool use_graph = true;
  int spmv_group = 0;         // Bsr::group of every level's A, P and R
  // the finest level's assembled node stencil (slot-major, A's block size; the
  // FP32 copy in the layout stf_node_major names): when given, the Lanczos
  // estimate of that level applies it instead of the BSR copy
  MeshDev mesh{};
  const double* st = nullptr;
  const float* stf = nullptr;
  bool stf_node_major = false;
};

// Build a hierarchy for the block matrix A (FP64 values, block size br) with
// near-null space B (n scalar rows x nns columns, column-major).  A is copied.
void amg_build(Amg& amg, const Bsr& A, const double* B, int nns, const AmgParams& prm,
               cudaStream_t s);
// z = V-cycle(r) (FP64 in / out; the cycle runs in FP32 when amg.mixed).
void amg_vcycle(Amg& amg, const double* r, double* z, cudaStream_t s);

// ---------------------------------------------------------------- linalg ---
// Deterministic two-pass reductions: the result lands in a device double.
void dot_dev(const double* x, const double* y, int64_t n, double* out, double* partials,
             cudaStream_t s);
void nrm_inf_dev(const double* x, int64_t n, double* out, double* partials, cudaStream_t s);
// <x, y> of FP32 vectors (FP32 products per thread, FP64 sums beyond)
void dot_dev_f32(const float* x, const float* y, int64_t n, double* out, double* partials,
                 cudaStream_t s);
// Fused: out[k] = <V_k, w> for k < nv (V stored as nv vectors of stride ld).
void multidot_dev(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* out,
                  double* partials, cudaStream_t s);
// w -= sum_k h[k] V_k   (h on device)
// Gram-Schmidt with FP32 coefficients (mixed precision): out[k] = <Vf_k, w>
// (k < nv; Vf the f32_view of the basis), out[nv] = ||w||^2, from the f32_view
// of w; part holds (nv + 1) * GS_MAX_BLOCKS floats
void gs_dot_dev(const float* Vf, int64_t ld, int nv, const double* w, int64_t n, float* part,
                double* out, cudaStream_t s);
// w <- w - V h in FP64; *nrm2 = ||w_new||^2 (FP32 view); part holds GS_MAX_BLOCKS floats
void gs_axpy_dev(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n,
                 float* part, double* nrm2, cudaStream_t s);
int sm_count();
// L2 size of the current device in bytes (0 if unknown); first called outside
// any stream capture
int64_t l2_cache_bytes();
void multi_axpy_dev(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n,
                    double sign, cudaStream_t s);
void exclusive_scan_int(const int* in, int* out, int n, int* total_host, cudaStream_t s);

enum { RED_PARTIALS = 1024 };   // partial buffer length needed by the reductions
// mixed-precision Gram-Schmidt: rows staged per block, blocks per pass
enum { GS_MAX_ROWS = 8192, GS_MAX_BLOCKS = 4096 };

// BSR SpMV y = alpha A x + beta y (FP64 or FP32 values / vectors)
void bsr_spmv(const Bsr& A, const double* x, double* y, double alpha, double beta, cudaStream_t s);
void bsr_spmv_f(const Bsr& A, const float* x, float* y, float alpha, float beta, cudaStream_t s);
// r = rhs - A x (square blocks)
template <class T>
void bsr_resid(const Bsr& A, const T* rhs, const T* x, T* r, cudaStream_t s);
// one Chebyshev step: d = cd d + cr dinv (rhs - A xin); xout = xin + d (zero_x: xin = d = 0)
template <class T>
void bsr_cheb(const Bsr& A, const T* dinv, const T* rhs, const T* xin, T* xout, T* d, T cd, T cr,
              bool zero_x, cudaStream_t s);
int bsr_group(const Bsr& A);
// algorithmic bytes of one SpMV with A (elem-byte values; beta: y is read too)
double bsr_bytes(const Bsr& A, int elem, bool beta);
enum { BSR_SELL = 64 };
// build (or rebuild) the SELL-32 copy of A's FP32 values
void bsr_make_sell(Bsr& A, cudaStream_t s);
// time the lane-group widths of the vector kernels on A (FP32 or FP64 values)
// and store the fastest in A.group (cached per matrix class)
void bsr_autotune(Bsr& A, bool f32, cudaStream_t s);

// ------------------------------------------------------------ FE kernels ---
struct Material {
  double E, nu, Gc, kappa, eps, p, mu, lam;
};

// stencil slot count and layout helpers
inline int n_slots(int dim) { return dim == 2 ? 9 : 27; }

void launch_phi_tilde(const MeshDev& m, int64_t n, int steps_done, const double* phi_old,
                      const double* phi_prev, double* phit, cudaStream_t s);
void launch_lumped_mass(const MeshDev& m, int64_t n, double* mass, cudaStream_t s);
// Per-cell quadrature records shared by the residual and the phase-field
// assembly (doubles for a mesh of n_cells cells).
int64_t qp_doubles(int dim, int64_t n_cells);
void launch_residual(const MeshDev& m, const Material& mat, int64_t n, int64_t n_cells,
                     const double* u, const double* phi, const double* phit, double* qp,
                     double* F, cudaStream_t s);
void launch_assemble_uu(const MeshDev& m, const Material& mat, int64_t n, const double* phit,
                        double* Kuu, cudaStream_t s);
void launch_assemble_phi(const MeshDev& m, const Material& mat, int64_t n, int64_t n_cells,
                         const double* u, const double* phi, double* qp, double* Kpu, double* Kpp,
                         cudaStream_t s);
// scaling S (u: diag M_uu, Dirichlet 1; phi: diag G_c(M/eps + eps K)) and its inverse
void launch_scaling(const MeshDev& m, const Material& mat, int64_t n, const double* Kuu,
                    double* S, double* Sinv, cudaStream_t s);
// reduced rhs: Ft = F with Dirichlet rows 0, active phi rows 0 and the active
// columns (dphiA = phi_old - phi on the active set) moved to the rhs; masks the
// phi rows / cols of Kpu, Kpp for the active set; writes dUA.
void launch_reduce_phi(const MeshDev& m, int64_t n, const uint8_t* active, const double* phi,
                       const double* phi_old, const double* F, double* Ft, double* dUA,
                       double* Kpu, double* Kpp, cudaStream_t s);
// y = Sinv .* (G~ x) with the assembled stencils (Sinv may be null)
void launch_apply_assembled(const MeshDev& m, int64_t n, const double* Kuu, const double* Kpu,
                            const double* Kpp, const double* x, double* y, const double* Sinv,
                            cudaStream_t s);
// y = Sinv .* (G~ x) matrix-free (Sinv may be null)
void launch_apply_matfree(const MeshDev& m, const Material& mat, int64_t n, const double* u,
                          const double* phi, const double* phit, const uint8_t* active,
                          const double* x, double* y, const double* Sinv, cudaStream_t s);
// Active set (step 2 of the Section 3 algorithm) with cycle locking:
// A = {indicator > tau} plus locked indices.  counters[0] = |A|, counters[1] =
// changes vs. the previous A (if have_prev), counters[3] = locked indices.
void launch_active_set(int64_t n, int dim, const double* F, const double* mass, const double* phi,
                       const double* phi_old, double c, double tau, double band, int have_prev,
                       int lock_after,
                       uint8_t* raw_prev, int* toggles, uint8_t* locked, uint8_t* active,
                       double* indicator, int* counters, cudaStream_t s);


// rho = Sinv .* F on free rows (not Dirichlet, not active), 0 elsewhere
void launch_scaled_reduced(const MeshDev& m, int64_t n, const double* F, const double* Sinv,
                           const uint8_t* active, double* rho, cudaStream_t s);
// stencil -> BSR value copy (structure precomputed)
void launch_stencil_to_bsr(const MeshDev& m, int64_t n, int b, const double* K, const Bsr& A,
                           cudaStream_t s);
void build_stencil_bsr_structure(const MeshDev& m, int64_t n, int b, Bsr& A, cudaStream_t s);
// rigid-body (u) near-null space, column-major n*dim x nns
void launch_rigid_modes(const MeshDev& m, int64_t n, double* B, cudaStream_t s);
// node coordinates [n][dim]
void launch_node_coords(const MeshDev& m, int64_t n, double* xyz, cudaStream_t s);
// AMG finest level on the node stencil (T = float or double; b = dim or 1).
// FP64: the full slot-major stencil.  FP32: the symmetric half (centre slot
// and the slots after it, stencil_to_f32 / stencil_to_node_major); node_major:
// K is the node-major copy of a 2d displacement stencil, otherwise slot-major
// with slot stride n
// rhs64 (with rhs_store): take the right-hand side from an FP64 vector and store
// its T copy; out64: write x_out in FP64 there instead of x_out and d.
template <class T>
void launch_stencil_cheb(const MeshDev& m, int64_t n, int b, const T* K, const T* dinv,
                         const T* rhs, const T* xin, T* xout, T* d, double cd, double cr,
                         int zero_x, cudaStream_t s, bool node_major = false,
                         const double* rhs64 = nullptr, T* rhs_store = nullptr,
                         double* out64 = nullptr);
template <class T>
void launch_stencil_resid(const MeshDev& m, int64_t n, int b, const T* K, const T* rhs, const T* x,
                          T* r, cudaStream_t s, bool node_major = false);
// FP32 node-major copy Kq[(h n + i) * 4 + 2a + c], slot s = h + 4, of the
// symmetric half of a 2d displacement stencil (5 n float4)
void stencil_to_node_major(const double* K, float* Kq, int64_t n, cudaStream_t s);
// FP32 slot-major copy of the symmetric half of a stencil of block size b
// (stencil_f32_count floats)
int64_t stencil_f32_count(int dim, int b, int64_t n);
void stencil_to_f32(int dim, int b, const double* K, float* Kf, int64_t n, cudaStream_t s);
void convert_d2f(const double* a, float* b, int64_t n, cudaStream_t s);
// dinv (and its FP32 copy, may be null) = inverse diagonal of a node stencil
void launch_stencil_dinv(const MeshDev& m, int64_t n, int b, const double* K, double* dinv,
                         float* dinvf, cudaStream_t s);
// TCV partial sums (deterministic) and COD line integrals
void tcv_dev(const MeshDev& m, int64_t n_cells, const double* u, const double* phi, double* out,
             double* partials, cudaStream_t s);
struct CodColumn {
  int col[2];       // cell index along x (and y in 3d)
  double xi[2];     // local coordinate in that cell
  double w;         // averaging weight
  int point;        // output slot
};
void cod_dev(const MeshDev& m, const CodColumn* cols, int ncols, const double* u,
             const double* phi, double* out, int npts, cudaStream_t s);
// adaptive refinement (Section 3, refinement strategy): gradient-jump indicator
// eta_K^2 per cell; per axis slab the sum of eta2 and the smallest nodal phi
// (slabs of all axes numbered consecutively); Q1 transfer of a nodal field
// (ncomp values per node) given each new axis coordinate's source interval and
// local coordinate
void jump_indicator_dev(const MeshDev& m, int64_t n_cells, const double* u, double* eta2,
                        cudaStream_t s);
void slab_reduce_dev(const MeshDev& m, const double* eta2, const double* phi, double* S,
                     double* minphi, cudaStream_t s);
void transfer_dev(int dim, const int* dst_nn, const int* src_nn, const int* const* cell,
                  const double* const* t, const double* src, int ncomp, double* dst,
                  cudaStream_t s);

}  // namespace pff

// -------------------------------------------------------------- the handle --
struct pff_problem {
  int dim = 2;
  int nn[3] = {1, 1, 1}, nc[3] = {1, 1, 1};
  int64_t n_nodes = 0, n_cells = 0, n_dofs = 0;
  std::vector<double> hX[3];
  double* X[3] = {nullptr, nullptr, nullptr};
  pff::Material mat{1.0, 0.2, 1.0, 1e-10, 0.0625, 0.0, 0.0, 0.0};
  cudaStream_t stream = nullptr;
  // second stream of the block preconditioner: the phase-field V-cycle runs on
  // it while the displacement V-cycle runs on `stream` (fork / join by events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool overlap = true;

  // state (device)
  double *u = nullptr, *phi = nullptr, *phi_old = nullptr, *phi_prev = nullptr, *phit = nullptr;
  int steps_done = 0;
  double *mass = nullptr, *S = nullptr, *Sinv = nullptr;
  double *Sw = nullptr, *Sinvw = nullptr;           // block-balanced scaling of a Newton solve
  const double *op_S = nullptr, *op_Sinv = nullptr;  // scaling FGMRES uses (null: S, Sinv)
  uint8_t *active = nullptr, *active_prev = nullptr, *raw_prev = nullptr, *locked = nullptr;
  int* toggles = nullptr;
  double* indicator = nullptr;
  int* counters = nullptr;      // device ints
  int* h_counters = nullptr;    // pinned host mirror
  double* h_scalars = nullptr;  // pinned host doubles
  double* d_scalars = nullptr;  // device doubles
  double* partials = nullptr;

  // assembled stencils
  double *Kuu = nullptr, *Kpu = nullptr, *Kpp = nullptr;
  float *Kuu_f = nullptr, *Kpp_f = nullptr;   // FP32 copies for the mixed-precision AMG
  bool uu_assembled = false, phi_assembled = false;

  // work vectors (n_dofs)
  double *F = nullptr, *Ft = nullptr, *dU = nullptr, *dUA = nullptr;
  double *ut = nullptr, *phit_trial = nullptr, *Ftrial = nullptr;
  bool F_ready = false;   // F already holds the residual of the current (u, phi), p, phi~

  // preconditioner
  pff::Bsr Auu, App;
  double* xyz = nullptr;  // node coordinates [n][dim] (AMG distance strength)
  double* Bu = nullptr;   // rigid-body modes
  double* Bp = nullptr;   // constants
  pff::Amg amg_u, amg_p;
  bool amg_u_valid = false;      // false: the displacement hierarchy must be rebuilt
  bool amg_u_check = false;      // a new loading step: compare phi~ with phit_built
  double* phit_built = nullptr;  // phi~ the displacement hierarchy was built from
  int amg_u_age = 0;             // loading steps the displacement hierarchy was reused for
  // the phase-field hierarchy is reused while the active set barely moves
  bool amg_p_valid = false;      // false: the phase-field hierarchy must be rebuilt
  uint8_t* active_built = nullptr;  // active set the phase-field hierarchy was built for
  int phi_amg_age = 0;           // Newton iterations since the last build
  double rho_last = 0.0;         // scaled reduced residual of the previous Newton iteration
  int precision = PFF_PREC_FP64;

  // Krylov workspace
  int krylov_m = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *h = nullptr, *tmp = nullptr;
  float* gs_part = nullptr;   // partial sums of the mixed-precision Gram-Schmidt
  float* Vf = nullptr;        // f32_view of the Krylov basis (mixed Gram-Schmidt)
  double* pc_tmp = nullptr;   // work vector of the block lower-triangular preconditioner
  double* qp = nullptr;       // per-cell quadrature records (residual, phase-field assembly)
  // one FGMRES iteration's device work (preconditioner + Jacobian apply) as a
  // CUDA graph on fixed buffers, for problems small enough to be launch-bound
  cudaGraphExec_t iter_graph = nullptr;
  int iter_graph_kernels = 0;
  double *g_in = nullptr, *g_out = nullptr;
  uint64_t iter_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double* h_host = nullptr;

  // Newton step state
  bool in_step = false;
  bool have_prev = false;
  bool last_small = false;
  int k = 0;
  double rho0 = 0.0;
  int apply_variant = PFF_APPLY_ASSEMBLED;
  bool apply_auto = false;         // PFF_APPLY_AUTO requested: time both applies once
  bool apply_tuned = false;
  pff_step_report cur{};

  pff::MeshDev mesh() const {
    pff::MeshDev m;
    m.dim = dim;
    for (int a = 0; a < 3; ++a) {
      m.nn[a] = nn[a];
      m.nc[a] = nc[a];
      m.X[a] = X[a];
    }
    return m;
  }
};

namespace pff {
// solver.cu
void begin_loading_step(pff_problem* P, double p);
int newton_iteration(pff_problem* P, const pff_options& o, pff_step_report* rep);
void end_loading_step(pff_problem* P);
void compute_residual(pff_problem* P, const double* u, const double* phi, double* F);
// a problem created with its set-up work and memory ordered on `stream`
pff_problem* create_problem(int dim, const int32_t* n_cells, const double* const* axis_coords,
                            cudaStream_t stream);
void compute_active_set(pff_problem* P, double c_rel, double tol_active, double tol_change,
                        int lock_after, bool track);
void assemble_all(pff_problem* P);
void precond_setup(pff_problem* P, const pff_options& o, bool allow_reuse = false);
void precond_apply(pff_problem* P, const double* r, double* z);
int fgmres(pff_problem* P, const pff_options& o, const double* b, double* x, int* iters);
void apply_jacobian(pff_problem* P, int variant, const double* x, double* y, const double* Sinv);
void ensure_krylov(pff_problem* P, int m);
void scale_into(const double* s, const double* x, double* y, int64_t n, cudaStream_t st);
// COD line descriptors of n_pts points (x in 2d; (x, y) pairs in 3d): the cells each
// line crosses, a line on a mesh line split between the two adjacent cells with
// weight 1/2 each (capi.cu; shared by both TCV / COD entry points)
std::vector<CodColumn> cod_columns(const pff_problem* P, int n_pts, const double* pts);
}  // namespace pff
