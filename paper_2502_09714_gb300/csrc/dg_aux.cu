// Auxiliary kernels of libdg: state conversion between the ABI layout and the
// internal layout, point-source injection and receiver sampling.
#include <cstdint>

#include "dg_internal.h"

namespace dg {
namespace {

// The conversions give each element copy one warp: it reads the copy's row in the source
// layout with coalesced loads into its own shared-memory row, and writes the row in the
// destination layout with coalesced stores.
constexpr int kConvWarps = 8;

// internal q[v][l*10+p] <- ABI src[m][e][p][l], v = e*M + m
template <int L>
__global__ void __launch_bounds__(32 * kConvWarps) k_state_in(int64_t E, int M, const void* src,
                                                              int src_is_double, float* q, int qs) {
  constexpr int R = kFields * L;
  __shared__ float t[kConvWarps][R];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t v = static_cast<int64_t>(blockIdx.x) * kConvWarps + wp;
  if (v >= E * M) return;
  const int64_t e = v / M, m = v - e * M;
  const int64_t base = (m * E + e) * R;
  float* tw = t[wp];
#pragma unroll
  for (int r = lane; r < R; r += 32)
    tw[r] = src_is_double ? static_cast<float>(static_cast<const double*>(src)[base + r])
                          : static_cast<const float*>(src)[base + r];
  __syncwarp();
  float* qv = q + v * qs;
#pragma unroll
  for (int w = lane; w < round4(R); w += 32) {
    float val = 0.f;
    if (w < R) {
      const int k = w / kFields, p = w - k * kFields;
      val = tw[p * L + k];
    }
    if (w < qs) qv[w] = val;
  }
}

// ABI dst[m][e][p][l] <- internal q[v], v = e*M + m
template <int L>
__global__ void __launch_bounds__(32 * kConvWarps) k_state_out(int64_t E, int M, const float* q, int qs,
                                                               void* dst, int dst_is_double) {
  constexpr int R = kFields * L;
  __shared__ float t[kConvWarps][R];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t v = static_cast<int64_t>(blockIdx.x) * kConvWarps + wp;
  if (v >= E * M) return;
  const int64_t e = v / M, m = v - e * M;
  const int64_t base = (m * E + e) * R;
  float* tw = t[wp];
  const float* qv = q + v * qs;
#pragma unroll
  for (int r = lane; r < R; r += 32) tw[r] = qv[r];
  __syncwarp();
#pragma unroll
  for (int w = lane; w < R; w += 32) {
    const int p = w / L, l = w - p * L;
    const float val = tw[l * kFields + p];
    if (dst_is_double) static_cast<double*>(dst)[base + w] = static_cast<double>(val);
    else static_cast<float*>(dst)[base + w] = val;
  }
}

// Sources whose element copy lies in [e_lo, e_hi) (all of them for the full range).
__global__ void k_sources(int L, int qs, int n_src, const SourceDev* src, const float* amp, int64_t step, float* q,
                          int64_t e_lo, int64_t e_hi) {
  const int s = blockIdx.x;
  if (s >= n_src) return;
  const int64_t e = src[s].elem;
  if (e < e_lo || e >= e_hi) return;
  const float a = amp[step * n_src + s];
  for (int w = threadIdx.x; w < 6 * L; w += blockDim.x) {
    const int p = w / L, l = w % L;
    atomicAdd(&q[e * qs + l * kFields + p], -a * src[s].phi_eps[p * L + l]);
  }
}

__global__ void k_receivers(int L, int qs, int n_rec, const ReceiverDev* rec, const float* q, float* out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= 3 * n_rec) return;
  const int r = w / 3, m = w % 3;
  const int64_t e = rec[r].elem;
  float v = 0.f;
  for (int l = 0; l < L; ++l) v += rec[r].phi[l] * q[e * qs + l * kFields + 6 + m];
  out[w] = v;
}

template <int N>
cudaError_t state_in_t(int64_t E, int M, const void* src, int dbl, float* q, cudaStream_t s) {
  const int64_t blocks = (E * M + kConvWarps - 1) / kConvWarps;
  if (blocks == 0) return cudaSuccess;
  k_state_in<n_modes(N)><<<static_cast<unsigned>(blocks), 32 * kConvWarps, 0, s>>>(E, M, src, dbl, q, q_stride(N));
  return cudaGetLastError();
}

template <int N>
cudaError_t state_out_t(int64_t E, int M, const float* q, void* dst, int dbl, cudaStream_t s) {
  const int64_t blocks = (E * M + kConvWarps - 1) / kConvWarps;
  if (blocks == 0) return cudaSuccess;
  k_state_out<n_modes(N)><<<static_cast<unsigned>(blocks), 32 * kConvWarps, 0, s>>>(E, M, q, q_stride(N), dst, dbl);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_state_in(int N, int64_t E, int M, const void* src, int dbl, float* q, cudaStream_t s) {
  switch (N) {
    case 1: return state_in_t<1>(E, M, src, dbl, q, s);
    case 2: return state_in_t<2>(E, M, src, dbl, q, s);
    case 3: return state_in_t<3>(E, M, src, dbl, q, s);
    case 4: return state_in_t<4>(E, M, src, dbl, q, s);
    case 5: return state_in_t<5>(E, M, src, dbl, q, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_state_out(int N, int64_t E, int M, const float* q, void* dst, int dbl, cudaStream_t s) {
  switch (N) {
    case 1: return state_out_t<1>(E, M, q, dst, dbl, s);
    case 2: return state_out_t<2>(E, M, q, dst, dbl, s);
    case 3: return state_out_t<3>(E, M, q, dst, dbl, s);
    case 4: return state_out_t<4>(E, M, q, dst, dbl, s);
    case 5: return state_out_t<5>(E, M, q, dst, dbl, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sources(int N, int n_src, const SourceDev* src, const float* amp, int64_t step,
                           float* q, cudaStream_t s) {
  k_sources<<<n_src, 128, 0, s>>>(n_modes(N), q_stride(N), n_src, src, amp, step, q, 0, INT64_MAX);
  return cudaGetLastError();
}

cudaError_t launch_sources_range(int N, int n_src, const SourceDev* src, const float* amp, int64_t step,
                                 float* q, int64_t e_lo, int64_t e_hi, cudaStream_t s) {
  k_sources<<<n_src, 128, 0, s>>>(n_modes(N), q_stride(N), n_src, src, amp, step, q, e_lo, e_hi);
  return cudaGetLastError();
}

cudaError_t launch_receivers(int N, int n_rec, const ReceiverDev* rec, const float* q, float* out,
                             cudaStream_t s) {
  const int threads = 3 * n_rec;
  k_receivers<<<(threads + 127) / 128, 128, 0, s>>>(n_modes(N), q_stride(N), n_rec, rec, q, out);
  return cudaGetLastError();
}

}  // namespace dg
