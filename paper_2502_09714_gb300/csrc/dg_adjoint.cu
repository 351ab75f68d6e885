// Instantiations of the adjoint kernels (dg_adjoint.cuh) for the compiled
// degrees, and the receiver-misfit kernel of the adjoint's seed.
#include "dg_adjoint.cuh"

namespace dg {

template cudaError_t launch_adjoint_t<1>(const AdjArgs&, cudaStream_t);
template cudaError_t launch_adjoint_t<2>(const AdjArgs&, cudaStream_t);
template cudaError_t launch_adjoint_t<3>(const AdjArgs&, cudaStream_t);
template cudaError_t launch_adjoint_t<4>(const AdjArgs&, cudaStream_t);
template cudaError_t launch_adjoint_t<5>(const AdjArgs&, cudaStream_t);

cudaError_t launch_adjoint(int N, const AdjArgs& a, cudaStream_t s) {
  switch (N) {
    case 1: return launch_adjoint_t<1>(a, s);
    case 2: return launch_adjoint_t<2>(a, s);
    case 3: return launch_adjoint_t<3>(a, s);
    case 4: return launch_adjoint_t<4>(a, s);
    case 5: return launch_adjoint_t<5>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

namespace {
// One thread per (receiver, component): the velocity at the receiver from the
// modal state, its residual against the reference, the misfit term in FP64 and
// the adjoint source dt phi_l(xi_r) res on the element's velocity modes.
__global__ void k_misfit(int L, int QS, int n_rec, const ReceiverDev* rec, const float* q, const float* ref,
                         float dt, double* J, float* lam) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= 3 * n_rec) return;
  const int r = w / 3, c = w - 3 * r;
  const int64_t e = rec[r].elem;
  float v = 0.f;
  for (int l = 0; l < L; ++l) v = fmaf(rec[r].phi[l], q[e * QS + l * 10 + 6 + c], v);
  const float res = v - ref[w];
  atomicAdd(J, 0.5 * static_cast<double>(dt) * static_cast<double>(res) * static_cast<double>(res));
  for (int l = 0; l < L; ++l) atomicAdd(lam + e * QS + l * 10 + 6 + c, dt * rec[r].phi[l] * res);
}
}  // namespace

cudaError_t launch_misfit(int N, int n_rec, const ReceiverDev* rec, const float* q, const float* ref, float dt,
                          double* J, float* lam, cudaStream_t s) {
  if (n_rec <= 0) return cudaSuccess;
  const int n = 3 * n_rec;
  k_misfit<<<(n + 127) / 128, 128, 0, s>>>(n_modes(N), q_stride(N), n_rec, rec, q, ref, dt, J, lam);
  return cudaGetLastError();
}

}  // namespace dg
