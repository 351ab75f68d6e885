// Internal declarations shared by the host runtime (dg_host.cpp) and the CUDA
// kernels (dg_step_n*.cu, dg_aux.cu).  Not part of the public C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dg {

constexpr int kFields = 10;      // eps_xx eps_yy eps_zz eps_xy eps_yz eps_zx v_x v_y v_z alpha
constexpr int kWave = 9;         // fields that take part in the wave (flux) part
constexpr int kMaxOrder = 5;

__host__ __device__ constexpr int n_modes(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
__host__ __device__ constexpr int n_vol_nodes(int N) { return (N + 1) * (N + 1) * (N + 1); }
__host__ __device__ constexpr int n_face_nodes(int N) { return (N + 1) * (N + 1); }
__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

// Per-element state stride (floats): modal coefficients stored [L][10].
__host__ __device__ constexpr int q_stride(int N) { return round4(kFields * n_modes(N)); }

// Per-element predictor output: for i = 1..N the time derivative D^i of the 9
// wave fields restricted to the modes of degree <= N-i ([L_{N-i}][9] each),
// then D^1 of alpha on all L modes.
__host__ __device__ constexpr int d_offset(int N, int i) {
  int off = 0;
  for (int j = 1; j < i; ++j) off += kWave * n_modes(N - j);
  return off;
}
__host__ __device__ constexpr int d_alpha_offset(int N) { return d_offset(N, N + 1); }
__host__ __device__ constexpr int d_stride(int N) { return round4(d_alpha_offset(N) + n_modes(N)); }

__host__ __device__ constexpr int round2(int x) { return (x + 1) & ~1; }

// Padded sizes: LP modes (multiple of 4), NQP volume nodes and NFP face nodes
// (multiples of 2, for two-node register tiles).
__host__ __device__ constexpr int lp_of(int N) { return round4(n_modes(N)); }
__host__ __device__ constexpr int nqp_of(int N) { return round2(n_vol_nodes(N)); }
__host__ __device__ constexpr int nfp_of(int N) { return round2(n_face_nodes(N)); }
__host__ __device__ constexpr int round8(int x) { return (x + 7) & ~7; }

// Tensor-core volume evaluation (degrees 2..4, volume nodes <= 128): the basis
// values at the volume nodes as a 128 x KP operand (KP = L rounded up to 8) in
// the canonical K-major layout without swizzle (core matrices of 8 rows x 4
// elements, 128 bytes; consecutive along K, then 8-row groups), split into a
// TF32 high part and an FP32 remainder.
__host__ __device__ constexpr bool tc_volume(int N) { return N >= 2 && N <= 4; }
// K extent (volume nodes rounded up to 32) of the tensor-core projection, whose
// A operand w_q phi_l(x_q) sits in tensor memory: lane l, column q.
__host__ __device__ constexpr int tc_kq(int N) { return (n_vol_nodes(N) + 31) / 32 * 32; }
__host__ __device__ constexpr int tc_kp(int N) { return round8(n_modes(N)); }
__host__ __device__ constexpr int tc_canon(int row, int k, int kp) {
  return (row >> 3) * (kp / 4 * 32) + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

// Reference tables of degree N (FP32, one device buffer), offsets in floats.
// Padding entries are zero; every table starts on a 16-byte boundary.
struct TableLayout {
  int VvT;    // [L][NQP]    phi_l at volume node q
  int Vw;     // [NQ][LP]    w_q phi_k(x_q)            (volume weights sum to 1/6)
  int Gw;     // [3][NQ][LP] w_q d phi_k / d xi_e (x_q)
  int KtA;    // [3][L][LP]  KtA[e][l][k] = int phi_k d phi_l / d xi_e
  int KtB;    // [3][L][LP]  KtB[e][l][k] = int phi_l d phi_k / d xi_e
  int VfT;    // [4][L][NFP] phi_l at face node i of local face f
  int Vfw;    // [4][NF][LP] beta_i phi_k(x_i) at face node i of local face f (beta sums to 1)
  int PhiH;   // [128 x KP]  canonical tensor-core operand: TF32 part of phi_l(x_q) (rows q >= NQ zero)
  int PhiL;   // [128 x KP]  phi_l(x_q) minus its TF32 part, rounded to TF32
  int PrjH;   // [128][KQ]   TF32 part of w_q phi_l(x_q), row l, column q (zero beyond L and NQ)
  int PrjL;   // [128][KQ]   w_q phi_l(x_q) minus its TF32 part, rounded to TF32
  int PrjS;   // [LP]        sum_q w_q phi_l(x_q), summed in double
  int tz;     // [NT]        time nodes in [0,1]
  int gz;     // [NT]        time weights (sum 1)
  int Tfit;   // [NT][NT]    Tfit[j][z]: the inverse of tz_z^j / j!, the Taylor coefficients at
              //             t = 0 of the polynomial through values at the time nodes
  int total;
};

__host__ __device__ constexpr TableLayout table_layout(int N) {
  TableLayout t{};
  const int L = n_modes(N), NQ = n_vol_nodes(N), NF = n_face_nodes(N), NT = N + 1;
  const int LP = lp_of(N), NQP = nqp_of(N), NFP = nfp_of(N);
  int o = 0;
  t.VvT = o; o = round4(o + L * NQP);
  t.Vw = o;  o = round4(o + NQ * LP);
  t.Gw = o;  o = round4(o + 3 * NQ * LP);
  t.KtA = o; o = round4(o + 3 * L * LP);
  t.KtB = o; o = round4(o + 3 * L * LP);
  t.VfT = o; o = round4(o + 4 * L * NFP);
  t.Vfw = o; o = round4(o + 4 * NF * LP);
  t.PhiH = o; o = round4(o + (tc_volume(N) ? 128 * tc_kp(N) : 0));
  t.PhiL = o; o = round4(o + (tc_volume(N) ? 128 * tc_kp(N) : 0));
  t.PrjH = o; o = round4(o + (tc_volume(N) ? 128 * tc_kq(N) : 0));
  t.PrjL = o; o = round4(o + (tc_volume(N) ? 128 * tc_kq(N) : 0));
  t.PrjS = o; o = round4(o + (tc_volume(N) ? LP : 0));
  t.tz = o;  o += NT;
  t.gz = o;  o += NT;
  t.Tfit = o; o += NT * NT;
  t.total = round4(o);
  return t;
}

// Per-element geometry (32 floats).  The element's vertices are reordered by
// increasing global vertex id inside the library, so both sides of every face
// parametrise it identically (face f = face opposite sorted vertex f, its
// vertices in ascending order).
struct GeomF {
  float tinv[9];      // Theta^{-1}[e][d] = d xi_e / d x_d  (row-major e, d)
  float inv_detj;     // 1 / |det J|
  float pad0[2];
  float face[4][4];   // outward unit normal (x, y, z) and |S_f| / |det J|
  float pad1[4];
};
static_assert(sizeof(GeomF) == 32 * sizeof(float), "GeomF layout");

// Per-element material (8 floats).
struct MatF {
  float rho, lam0, mu0, gamma_r, xi0, cd, rho_inv, pad;
};

// Status bits of the device status word.
enum : unsigned {
  kStatusNonFinite = 1u,
  kStatusNonHyperbolic = 2u,
  kStatusIndex = 4u,
  kStatusTimeout = 8u,      // a bounded wait on the tensor cores ran out
};

// Time-integrated Rusanov flux of every face at its NF nodes (9 wave fields),
// oriented with the outward normal of the face's first element.
__host__ __device__ constexpr int ff_stride(int N) { return round4(n_face_nodes(N) * kWave); }

struct StepArgs {
  int64_t E;
  int64_t F;              // number of faces
  const float* q_in;      // [E][q_stride]
  float* q_out;           // [E][q_stride]
  float* d;               // [E][d_stride]
  float* cp;              // [E] effective P speed of the cell mean (for the Rusanov C)
  float* ff;              // [F][ff_stride] face fluxes
  const GeomF* geom;      // [E]
  const MatF* mat;        // [E]
  const int* nbr;         // [E][4] (neighbour element << 2) | neighbour's local face
  const int4* faces;      // [F] (element 0, its local face, element 1, its local face)
  const int* elem_face;   // [E][4] (face id << 1) | side (side 1: flux sign reversed)
  const float* tables;    // table_layout(N)
  float dt;
  unsigned* status;
  int grid_pred, grid_face, grid_corr;   // persistent grid sizes (0: one CTA per tile)
  int law;                // pointwise law: 0 = CDM (Eq. "cdb-model"), 1 = IVM (Eq. "ivm-model"),
                          // 2 = nonlinear shear (Eq. "1d Riemann eqs")
  int has_boundary;       // nonzero when the mesh has absorbing or free-surface faces
  int picard_iters;       // Picard iterations after the CK predictor (0: the CK alone)
  int wait_limit;         // polls of a bounded wait on the tensor cores, when wait_limit_set
  int wait_limit_set;     // 0: the kernels' default limit
};

// Kernel launchers, one per compiled degree (dg_step_n<N>.cu), and their
// dispatch on the runtime degree (dg_host.cpp).
template <int N> cudaError_t launch_predictor_t(const StepArgs& a, cudaStream_t s);
template <int N> cudaError_t launch_faces_t(const StepArgs& a, cudaStream_t s);
template <int N> cudaError_t launch_corrector_t(const StepArgs& a, cudaStream_t s);
template <int N> cudaError_t launch_picard_t(const StepArgs& a, cudaStream_t s);
cudaError_t launch_predictor(int N, const StepArgs& a, cudaStream_t s);
cudaError_t launch_faces(int N, const StepArgs& a, cudaStream_t s);
cudaError_t launch_corrector(int N, const StepArgs& a, cudaStream_t s);
cudaError_t launch_picard(int N, const StepArgs& a, cudaStream_t s);

// Auxiliary kernels (dg_aux.cu).
// State conversion between the ABI layout [M][E][10][L] (FP64 or FP32) and the
// internal layout [E*M][q_stride] (copy e*M + m of element e for member m,
// [L][10] per copy, FP32).
cudaError_t launch_state_in(int N, int64_t E, int M, const void* src, int src_is_double, float* q,
                            cudaStream_t s);
cudaError_t launch_state_out(int N, int64_t E, int M, const float* q, void* dst, int dst_is_double,
                             cudaStream_t s);

struct SourceDev {
  int64_t elem;
  float phi_eps[6 * 64];   // phi_l(xi_s) * (C0^{-1}:M)_p / |J|, [6][L] (L <= 56)
};
// Adds -amp[step * n_src + s] * phi_eps to the strain modes of each source element.
cudaError_t launch_sources(int N, int n_src, const SourceDev* src, const float* amp, int64_t step,
                           float* q, cudaStream_t s);
// The sources whose element copy lies in [e_lo, e_hi).
cudaError_t launch_sources_range(int N, int n_src, const SourceDev* src, const float* amp, int64_t step,
                                 float* q, int64_t e_lo, int64_t e_hi, cudaStream_t s);

struct ReceiverDev {
  int64_t elem;
  float phi[64];           // phi_l(xi_r)
};
cudaError_t launch_receivers(int N, int n_rec, const ReceiverDev* rec, const float* q,
                             float* traces_row, cudaStream_t s);

// Discrete adjoint of one step (dg_adjoint.cu).  A face record holds, per face
// and side, lam of that side's D^0..D^N in the (Q, D) layout (q_stride floats of
// order 0, then d_stride floats of the higher orders) and four scalars: lam of the
// side's P speed and the xi0 part of the side's flux.
__host__ __device__ constexpr int adj_rec_stride(int N) { return q_stride(N) + d_stride(N) + 4; }
struct AdjArgs {
  int64_t E, F;           // elements, faces (interior first, then boundary)
  const float* q;         // Q^k [E][q_stride]
  const float* d;         // predictor output of Q^k [E][d_stride]
  const float* cp;        // effective P speeds of Q^k [E]
  const float* lam_in;    // dJ/dQ^{k+1} [E][q_stride]
  float* lam_out;         // dJ/dQ^k [E][q_stride]
  float* rec;             // [F][2][adj_rec_stride]
  double* g_xi0;          // [E] dJ/dxi0, accumulated
  double* g_cd;           // [E] dJ/dC_d, accumulated
  const GeomF* geom;
  const MatF* mat;
  const int4* faces;
  const int* elem_face;
  const float* tables;
  float dt;
};
template <int N> cudaError_t launch_adjoint_t(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint(int N, const AdjArgs& a, cudaStream_t s);
// Receiver misfit at one state: res = v_r(q) - ref[r] for every receiver and
// component; adds 0.5 dt res^2 to *J (FP64) and dt phi_l(xi_r) res to lam[e_r].
cudaError_t launch_misfit(int N, int n_rec, const ReceiverDev* rec, const float* q, const float* ref, float dt,
                          double* J, float* lam, cudaStream_t s);

// Read-only view of a context for the allocation-free step (dg_noalloc.cu).
struct NoAllocView {
  int N;
  int64_t E;              // element copies (mesh elements x members)
  int M;
  cudaStream_t stream;
  const GeomF* geom;
  const MatF* mat;
  const int* nbr;
  const int4* faces;
  const int* elem_face;
  int64_t F;
  bool has_boundary;
  const float* tables;
  double dt_cfl;
  bool has_material;
  int law;
  int picard_iters;
};

}  // namespace dg
