// dg_step_noalloc: one ADER-DG step that allocates no device or host memory.
//
// Some callers cannot call cudaMalloc while they step (a process held to a
// fixed device-memory budget, an embedding that forbids allocation after
// set-up).  This entry point keeps every intermediate of the step in one
// file-scope device array of fixed size instead of the context's buffers; the
// caller passes the input and output states.  The kernels are the same
// predictor, face-flux and corrector kernels as dg_step.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dg {
bool noalloc_view(const dg_ctx* ctx, NoAllocView* v);
dg_status noalloc_error(dg_ctx* ctx, dg_status s, const char* msg);
}  // namespace dg

namespace {

using namespace dg;

// 16 MiB of scratch, held by every GPU that loads the library until exit.
constexpr int64_t kScratchFloats = int64_t(4) << 20;
constexpr int64_t kStatusFloats = 64;   // status word, padded to 256 bytes
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

// In host code the array's name is only a host-side stand-in; its device
// address is looked up once per device, with that device current.
constexpr int kMaxDevices = 64;
float* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" dg_status dg_step_noalloc(dg_ctx* ctx, const float* q_in, float* q_out, double dt) {
  NoAllocView v{};
  if (!ctx || !noalloc_view(ctx, &v)) return noalloc_error(ctx, DG_E_ARG, "NULL context");
  if (!q_in || !q_out) return noalloc_error(ctx, DG_E_ARG, "NULL state pointer");
  if (!v.has_material) return noalloc_error(ctx, DG_E_STATE, "dg_set_material must precede dg_step_noalloc");
  if (v.M != 1) return noalloc_error(ctx, DG_E_UNSUPPORTED, "dg_step_noalloc takes one member only");
  if (dt <= 0) dt = v.dt_cfl;
  if (!std::isfinite(dt)) return noalloc_error(ctx, DG_E_ARG, "non-finite dt");
  const int64_t qs = q_stride(v.N), ds = d_stride(v.N), ffs = ff_stride(v.N);
  const int64_t cp_floats = (v.E + 3) / 4 * 4;
  const int64_t need = kStatusFloats + v.E * (2 * qs + ds) + cp_floats + v.F * ffs;
  if (need > kScratchFloats) {
    // a closed mesh has two faces per element
    const int64_t max_elem = (kScratchFloats - kStatusFloats - 3) / (2 * qs + ds + 1 + 2 * ffs);
    const std::string msg = "dg_step_noalloc: " + std::to_string(v.E) + " elements exceed the " +
                            std::to_string(max_elem) + "-element capacity of its 16 MiB static scratch at order " +
                            std::to_string(v.N);
    return noalloc_error(ctx, DG_E_ARG, msg.c_str());
  }
  float* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess)
    return noalloc_error(ctx, DG_E_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
  unsigned* status = reinterpret_cast<unsigned*>(base);
  float* qa = base + kStatusFloats;          // state in, internal layout (offsets keep 16-byte alignment)
  float* qb = qa + v.E * qs;                 // state out, internal layout
  float* d = qb + v.E * qs;                  // predictor output
  float* cp = d + v.E * ds;                  // effective P speed per cell
  float* ff = cp + cp_floats;                // face fluxes (16-byte aligned)
  StepArgs a{};
  a.E = v.E;
  a.F = v.F;
  a.has_boundary = v.has_boundary;
  a.ff = ff;
  a.faces = v.faces;
  a.elem_face = v.elem_face;
  a.q_in = qa;
  a.q_out = qb;
  a.d = d;
  a.cp = cp;
  a.geom = v.geom;
  a.mat = v.mat;
  a.nbr = v.nbr;
  a.tables = v.tables;
  a.dt = static_cast<float>(dt);
  a.status = status;
  a.law = v.law;
  a.picard_iters = v.picard_iters;
  // the array keeps the previous call's contents: the status word must start at zero
  if ((e = cudaMemsetAsync(status, 0, sizeof(unsigned), v.stream)) != cudaSuccess ||
      (e = launch_state_in(v.N, v.E, 1, q_in, 0, qa, v.stream)) != cudaSuccess ||
      (e = launch_predictor(v.N, a, v.stream)) != cudaSuccess ||
      (a.picard_iters > 0 && (e = launch_picard(v.N, a, v.stream)) != cudaSuccess) ||
      (e = launch_faces(v.N, a, v.stream)) != cudaSuccess ||
      (e = launch_corrector(v.N, a, v.stream)) != cudaSuccess ||
      (e = launch_state_out(v.N, v.E, 1, qb, q_out, 0, v.stream)) != cudaSuccess)
    return noalloc_error(ctx, DG_E_CUDA, (std::string("dg_step_noalloc launch: ") + cudaGetErrorString(e)).c_str());
  unsigned st = 0;
  if ((e = cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, v.stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(v.stream)) != cudaSuccess)
    return noalloc_error(ctx, DG_E_CUDA, (std::string("dg_step_noalloc: ") + cudaGetErrorString(e)).c_str());
  if (st & kStatusNonFinite) return noalloc_error(ctx, DG_E_NONFINITE, "non-finite value in the state");
  if (st & kStatusNonHyperbolic) return noalloc_error(ctx, DG_E_NONHYPERBOLIC, "effective moduli lost hyperbolicity");
  if (st & kStatusIndex) return noalloc_error(ctx, DG_E_MESH, "neighbour index out of range");
  if (st & kStatusTimeout) return noalloc_error(ctx, DG_E_CUDA, "a bounded wait on the tensor cores timed out");
  return DG_OK;
}
