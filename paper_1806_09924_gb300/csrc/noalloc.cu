// TCV / COD evaluation that performs no device allocation.
//
// pff_eval_tcv_cod allocates a small device buffer for the COD line
// descriptors on every call.  Some callers cannot let a library allocate
// device memory: an application whose device memory is all handed out by its
// own pool allocator, or one that has reserved the whole memory of the GPU up
// front, gets an out-of-memory error (or breaks its own accounting) from a
// cudaMalloc it did not plan for.  Those callers use pff_eval_tcv_cod_noalloc
// instead.  It runs the same TCV and COD kernels, but every piece of scratch
// they need (line descriptors, per-line sums, per-block TCV partial sums)
// lives in one file-scope device array of fixed size, loaded with the library
// and kept by every GPU that uses it until the process exits.  The call
// synchronizes the problem's stream before it returns (the results are copied
// to the caller's host memory).
#include <mutex>
#include <string>
#include <vector>

#include "pff_internal.h"

namespace pff {
namespace {

// Layout of the scratch array (units of 8 bytes):
//   [0, kColDoubles)                   line descriptors (CodColumn)
//   [kColDoubles, +kMaxCols)           one integral per line
//   [.., +RED_PARTIALS)                per-block TCV partial sums
//   [.., +1)                           the TCV value
constexpr int kMaxCols = 4 * PFF_NOALLOC_MAX_POINTS;   // at most 4 lines per point (3d)
constexpr size_t kColDoubles = (sizeof(CodColumn) * kMaxCols + 7) / 8;
constexpr size_t kScratchDoubles = kColDoubles + kMaxCols + RED_PARTIALS + 1;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

// Device address of g_scratch on each device, looked up once per device.
std::mutex g_mu;
double* g_addr[64] = {nullptr};

double* scratch_address() {
  int dev = 0;
  PFF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(PFF_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    PFF_CUDA(cudaGetSymbolAddress(&p, g_scratch));
    g_addr[dev] = static_cast<double*>(p);
  }
  return g_addr[dev];
}

}  // namespace
}  // namespace pff

extern "C" int pff_eval_tcv_cod_noalloc(pff_problem* P, int n_pts, const double* pts, double* tcv,
                                        double* cod) {
  API_BEGIN
  if (!P) pff::fail(PFF_ERR_INVALID_ARG, "problem is NULL");
  if (n_pts < 0 || (n_pts > 0 && !pts)) pff::fail(PFF_ERR_INVALID_ARG, "bad COD points");
  if (n_pts > PFF_NOALLOC_MAX_POINTS)
    pff::fail(PFF_ERR_CAPACITY, "pff_eval_tcv_cod_noalloc: " + std::to_string(n_pts) +
                                    " points exceed the fixed scratch limit of " +
                                    std::to_string(PFF_NOALLOC_MAX_POINTS));
  double* base = pff::scratch_address();
  auto* cols_dev = reinterpret_cast<pff::CodColumn*>(base);
  double* vals_dev = base + pff::kColDoubles;
  double* part_dev = vals_dev + pff::kMaxCols;
  double* tcv_dev = part_dev + pff::RED_PARTIALS;
  const auto m = P->mesh();
  cudaStream_t s = P->stream;
  if (tcv) {
    // every partial slot the final sum reads is written by this launch
    pff::tcv_dev(m, P->n_cells, P->u, P->phi, tcv_dev, part_dev, s);
    PFF_CUDA(cudaMemcpyAsync(tcv, tcv_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  if (cod && n_pts > 0) {
    // the same line descriptors as pff_eval_tcv_cod (at most 4 per point)
    const std::vector<pff::CodColumn> cols = pff::cod_columns(P, n_pts, pts);
    const int nc = (int)cols.size();
    std::vector<double> vals(nc);
    // each line's integral is written by its own block before it is read back
    PFF_CUDA(cudaMemcpyAsync(cols_dev, cols.data(), sizeof(pff::CodColumn) * nc,
                             cudaMemcpyHostToDevice, s));
    pff::cod_dev(m, cols_dev, nc, P->u, P->phi, vals_dev, n_pts, s);
    PFF_CUDA(cudaMemcpyAsync(vals.data(), vals_dev, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    PFF_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < n_pts; ++k) cod[k] = 0.0;
    for (int c = 0; c < nc; ++c) cod[cols[c].point] += vals[c];
  }
  PFF_CUDA(cudaStreamSynchronize(s));
  API_END
}
