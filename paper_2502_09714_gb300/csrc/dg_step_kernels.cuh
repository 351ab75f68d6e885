// Kernels of one ADER-DG step for the damage rheologies of arXiv 2502.09714
// (CDM of Eq. "cdb-model", IVM of Eq. "ivm-model"; Appendix A), FP32, templated
// on the degree N.
//
//   k_predictor_tc (degrees 2..4) / k_predictor (1, 5): cell-mean effective
//                Jacobian, Cauchy-Kovalevskaya recursion (Eq. "CKIter-ref-matrix")
//                and damage-rate source at i = 1 (Eq. "CKIter-ref-source") -> D, cp
//   k_face_flux  Rusanov flux (Eq. "rusanov-flux") of every interior face, once
//                per face, time-integrated (the stress at the space-time nodes,
//                the linear terms from the time-integrated trace); absorbing and
//                free-surface fluxes (Appendix A) on boundary faces -> FF
//   k_corrector_tc (degrees 2..4) / k_corrector (1, 5): volume flux and damage
//                source (Eqs. "3rd term", "rhs term"), face term (Eq. "2nd
//                term") from FF, update (Eq. "time-integrated")
//
// Each kernel is persistent: a CTA loads the reference tables it needs into
// shared memory once, then walks over tiles of elements (or faces).  For degrees
// 2..4 the evaluations at the volume nodes (the predictor's strains and alpha,
// the corrector's Taylor expansion, which feeds the pointwise law from tensor
// memory) and the corrector's projection run on the tensor cores (tcgen05,
// 3xTF32); the other contractions with the shared tables are block GEMMs with
// register tiles.
#pragma once

#include <algorithm>
#include <cstdlib>

#include "dg_internal.h"
#include "dg_tc.cuh"

namespace dg {

__host__ __device__ constexpr int sum_hi(int N) {
  int s = 0;
  for (int o = 1; o <= N; ++o) s += n_modes(N - o);
  return s;
}
// first row of Taylor order o >= 1 in the stacked higher-order arrays
__host__ __device__ constexpr int row_hi(int N, int o) {
  int s = 0;
  for (int j = 1; j < o; ++j) s += n_modes(N - j);
  return s;
}

template <int N>
struct Dim {
  static constexpr int L = n_modes(N), NQ = n_vol_nodes(N), NF = n_face_nodes(N), NT = N + 1;
  static constexpr int LP = lp_of(N), NQP = nqp_of(N), NFP = nfp_of(N);
  static constexpr int QS = q_stride(N), DS = d_stride(N), AOFF = d_alpha_offset(N), FFS = ff_stride(N);
  static constexpr int SH = sum_hi(N);
};

// Row stride of the nodal terms [NQ][10 TE]: padded so that consecutive volume
// nodes (one per lane) do not fall on the same banks.
__host__ __device__ constexpr int nb_stride(int te) { return 10 * te % 8 == 0 ? 10 * te + 4 : 10 * te; }

// CDM stress (Eq. "cdb-model") and damage rate, with xi = 0 below I2 = 1e-30
// and the rate written as C_d gamma_r max(0, I1 sqrt(I2) - xi0 I2).
__device__ __forceinline__ void cdm_point(const float e[6], float alpha, const MatF& m,
                                          float sig[6], float* rate) {
  const float I1 = e[0] + e[1] + e[2];
  const float I2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] +
                   2.f * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
  float s = 0.f, xi = 0.f;
  if (I2 > 1e-30f) {
    const float rs = rsqrtf(I2);
    s = I2 * rs;
    xi = I1 * rs;
  }
  const float ag = alpha * m.gamma_r;
  const float iso = m.lam0 * I1 - ag * s;
  const float sh = 2.f * (m.mu0 + ag * m.xi0) - ag * xi;
  sig[0] = iso + sh * e[0];
  sig[1] = iso + sh * e[1];
  sig[2] = iso + sh * e[2];
  sig[3] = sh * e[3];
  sig[4] = sh * e[4];
  sig[5] = sh * e[5];
  *rate = m.cd * m.gamma_r * fmaxf(0.f, I1 * s - m.xi0 * I2);
}

__device__ __forceinline__ float cdm_rate(const float e[6], const MatF& m) {
  const float I1 = e[0] + e[1] + e[2];
  const float I2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] +
                   2.f * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
  const float s = I2 > 1e-30f ? sqrtf(I2) : 0.f;
  return m.cd * m.gamma_r * fmaxf(0.f, I1 * s - m.xi0 * I2);
}

// IVM (Eq. "ivm-model" with l0 = m0 = n0 = 0): sigma = (1 - alpha)(lambda0 I1 delta
// + 2 mu0 eps) and r = (lambda0 I1^2/2 + mu0 I2 - gamma_b (alpha/(1-alpha))^2) /
// (gamma_b tau_b); the material holds gamma_b in gamma_r and 1/(gamma_b tau_b) in cd.
__device__ __forceinline__ void ivm_point(const float e[6], float alpha, const MatF& m, float sig[6],
                                          float* rate) {
  const float I1 = e[0] + e[1] + e[2];
  const float I2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + 2.f * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
  const float f = 1.f - alpha;
  const float iso = f * m.lam0 * I1, sh = 2.f * f * m.mu0;
  sig[0] = iso + sh * e[0];
  sig[1] = iso + sh * e[1];
  sig[2] = iso + sh * e[2];
  sig[3] = sh * e[3];
  sig[4] = sh * e[4];
  sig[5] = sh * e[5];
  const float s = alpha / f;
  *rate = m.cd * (0.5f * m.lam0 * I1 * I1 + m.mu0 * I2 - m.gamma_r * s * s);
}

// Nonlinear shear law of the 1-D Riemann verification (Eq. "1d Riemann eqs"):
// sigma = lambda0 I1 delta + 2 mu0 (1 - beta gamma) eps, gamma = sqrt(I2 / 2), which in
// plane shear is sigma_xy = 2 mu0 (1 - beta eps_xy) eps_xy for eps_xy >= 0; beta is
// held in gamma_r and alpha does not evolve.
__device__ __forceinline__ void nlshear_point(const float e[6], const MatF& m, float sig[6], float* rate) {
  const float I1 = e[0] + e[1] + e[2];
  const float I2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + 2.f * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
  const float sh = 2.f * m.mu0 * (1.f - m.gamma_r * sqrtf(0.5f * I2));
  const float iso = m.lam0 * I1;
  sig[0] = iso + sh * e[0];
  sig[1] = iso + sh * e[1];
  sig[2] = iso + sh * e[2];
  sig[3] = sh * e[3];
  sig[4] = sh * e[4];
  sig[5] = sh * e[5];
  *rate = 0.f;
}

// The pointwise law of the step: 0 = CDM, 1 = IVM, 2 = nonlinear shear.  Every law-
// dependent helper and kernel takes LAW: 0 compiles the CDM alone (the kernels run with
// it whenever the CDM is selected), -1 dispatches on the run-time value `law`.
template <int LAW>
__device__ __forceinline__ void law_point(int law, const float e[6], float alpha, const MatF& m, float sig[6],
                                          float* rate) {
  if constexpr (LAW == 0) {
    cdm_point(e, alpha, m, sig, rate);
  } else {
    if (law == 1) ivm_point(e, alpha, m, sig, rate);
    else if (law == 2) nlshear_point(e, m, sig, rate);
    else cdm_point(e, alpha, m, sig, rate);
  }
}
template <int LAW>
__device__ __forceinline__ float law_rate(int law, const float e[6], float alpha, const MatF& m) {
  if constexpr (LAW == 0) return cdm_rate(e, m);
  if (law == 2) return 0.f;
  if (law == 1) {
    float sig[6], r;
    ivm_point(e, alpha, m, sig, &r);
    return r;
  }
  return cdm_rate(e, m);
}

// Normal flux F^d(u) n_d of the 9 wave fields (Eq. "nonlinear hyper pdes"):
// strain rows -(v_i n_j + v_j n_i)/2, velocity rows -sigma_ij n_j / rho.
template <int LAW>
__device__ __forceinline__ void normal_flux(int law, const float u[10], const MatF& m, const float n[3], float F[9]) {
  float sig[6], r;
  law_point<LAW>(law, u, u[9], m, sig, &r);
  const float vx = u[6], vy = u[7], vz = u[8];
  F[0] = -vx * n[0];
  F[1] = -vy * n[1];
  F[2] = -vz * n[2];
  F[3] = -0.5f * (vx * n[1] + vy * n[0]);
  F[4] = -0.5f * (vy * n[2] + vz * n[1]);
  F[5] = -0.5f * (vz * n[0] + vx * n[2]);
  F[6] = -m.rho_inv * (sig[0] * n[0] + sig[3] * n[1] + sig[5] * n[2]);
  F[7] = -m.rho_inv * (sig[3] * n[0] + sig[1] * n[1] + sig[4] * n[2]);
  F[8] = -m.rho_inv * (sig[5] * n[0] + sig[4] * n[1] + sig[2] * n[2]);
}

// Effective Lame parameters at a cell mean (CDM: Eq. "effective-cdb" with the sign
// of the xi0 term taken from Eq. "cdb-model"; IVM: Eq. "effective-ivm"; nonlinear
// shear: the secant moduli); q0 holds the ten mode-0 coefficients.
template <int LAW>
__device__ __forceinline__ void effective_lame(int law, const float* q0, const MatF& m, float* lam, float* mu) {
  if constexpr (LAW == 0) law = 0;
  const float r6 = 2.449489742783178f;   // phi_0 = sqrt(6): cell mean = Q_0 sqrt(6)
  if (law == 1) {
    const float f = 1.f - q0[9] * r6;
    *lam = f * m.lam0;
    *mu = f * m.mu0;
    return;
  }
  float u[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) u[p] = q0[p] * r6;
  if (law == 2) {                        // secant moduli of the nonlinear shear law
    const float I2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + 2.f * (u[3] * u[3] + u[4] * u[4] + u[5] * u[5]);
    *lam = m.lam0;
    *mu = m.mu0 * (1.f - m.gamma_r * sqrtf(0.5f * I2));
    return;
  }
  const float alpha = q0[9] * r6;
  const float I1 = u[0] + u[1] + u[2];
  const float I2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + 2.f * (u[3] * u[3] + u[4] * u[4] + u[5] * u[5]);
  const float xi = I2 > 1e-30f ? I1 * rsqrtf(I2) : 0.f;
  *lam = m.lam0 - alpha * m.gamma_r * xi * (1.f / 3.f);
  *mu = m.mu0 + alpha * m.xi0 * m.gamma_r - 0.5f * alpha * m.gamma_r * xi;
}

// Normal flux on a boundary face (Appendix A, Eqs. "absorbing-flux" and
// "freeSurface-flux") written in global coordinates.  Characteristic analysis
// of the effective isotropic Jacobian along n gives, with the traction
// component sigma_nn = lambda I1 + 2 mu eps_nn, the tangential parts
// v_tan = v - (v.n) n and e_tan = eps n - eps_nn n,
//   a = -v.n + c_p sigma_nn / (lambda + 2 mu),   b = -v_tan / 2 + c_s e_tan:
// free surface (bc 1): strain flux a n n^T + n b^T + b n^T, velocity flux 0
//   (the boundary state is traction free);
// absorbing (bc 2): half that strain flux and the velocity flux
//   ((-sigma_nn / rho + c_p v.n) n + (-2 mu e_tan / rho + c_s v_tan)) / 2
//   (only the outgoing characteristics).
// k_p = c_p / (lambda + 2 mu).  The rotation into the face frame drops out, so
// no tangent vectors are needed.
__device__ __forceinline__ void boundary_flux(int bc, const float u[9], const float n[3], float lam, float mu,
                                              float rho_inv, float cp, float cs, float k_p, float F[9]) {
  const float En[3] = {u[0] * n[0] + u[3] * n[1] + u[5] * n[2], u[3] * n[0] + u[1] * n[1] + u[4] * n[2],
                       u[5] * n[0] + u[4] * n[1] + u[2] * n[2]};
  const float enn = En[0] * n[0] + En[1] * n[1] + En[2] * n[2];
  const float snn = lam * (u[0] + u[1] + u[2]) + 2.f * mu * enn;
  const float vn = u[6] * n[0] + u[7] * n[1] + u[8] * n[2];
  const float a = -vn + k_p * snn;
  float b[3], et[3], vt[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vt[i] = u[6 + i] - vn * n[i];
    et[i] = En[i] - enn * n[i];
    b[i] = -0.5f * vt[i] + cs * et[i];
  }
  const float h = bc == 2 ? 0.5f : 1.f;
  F[0] = h * (a * n[0] * n[0] + 2.f * n[0] * b[0]);
  F[1] = h * (a * n[1] * n[1] + 2.f * n[1] * b[1]);
  F[2] = h * (a * n[2] * n[2] + 2.f * n[2] * b[2]);
  F[3] = h * (a * n[0] * n[1] + n[0] * b[1] + b[0] * n[1]);
  F[4] = h * (a * n[1] * n[2] + n[1] * b[2] + b[1] * n[2]);
  F[5] = h * (a * n[2] * n[0] + n[2] * b[0] + b[2] * n[0]);
  if (bc == 2) {
    const float pn = 0.5f * (-snn * rho_inv + cp * vn);
#pragma unroll
    for (int i = 0; i < 3; ++i) F[6 + i] = pn * n[i] + 0.5f * (-2.f * mu * et[i] * rho_inv + cs * vt[i]);
  } else {
    F[6] = F[7] = F[8] = 0.f;
  }
}

__device__ __forceinline__ void copy_to_smem(float* dst, const float* src, int n) {
  for (int w = threadIdx.x; w < n; w += blockDim.x) dst[w] = __ldg(src + w);
}

// Block GEMM: C[m][n] = sum_k A[k*lda + m] B[k*ldb + n], m < M, n < Nc (both
// multiples of 4, rows 16-byte aligned), on threads t of [0, nt).  Work items are
// (m-quad, n-quad, k-split); out(m, n, value) receives each entry once.  With
// KS > 1 the split sums go through `partial` (KS*M*Nc floats) and the call runs
// bar() twice, so every one of the nt threads must make it.
template <int KS, int NJ = 4, class Out, class Bar>
__device__ __forceinline__ void block_gemm_part(const float* __restrict__ A, int lda,
                                                const float* __restrict__ B, int ldb, int M, int Nc,
                                                int K, float* partial, Out out, int t, int nt, Bar bar) {
  static_assert(NJ == 4 || NJ == 3 || NJ == 2, "4 rows x 4, 3 or 2 columns per work item");
  const int mq = M >> 2, nq = Nc / NJ, tiles = mq * nq;
  const int kchunk = (K + KS - 1) / KS;
  for (int w = t; w < tiles * KS; w += nt) {
    const int ks = w / tiles, r = w - ks * tiles;
    const int mi = r / nq, ni = r - mi * nq;   // column group fastest: the partial stores of a warp are contiguous
    float acc[4][NJ];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) acc[i][j] = 0.f;
    const int k0 = ks * kchunk;
    const int k1 = min(K, k0 + kchunk);
    const float* ap = A + 4 * mi;
    const float* bp = B + NJ * ni;
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(ap + k * lda);
      float bv[NJ];
      if constexpr (NJ == 4) {
        const float4 b = *reinterpret_cast<const float4*>(bp + k * ldb);
        bv[0] = b.x; bv[1] = b.y; bv[2] = b.z; bv[3] = b.w;
      } else if constexpr (NJ == 3) {
        bv[0] = bp[k * ldb]; bv[1] = bp[k * ldb + 1]; bv[2] = bp[k * ldb + 2];
      } else {
        const float2 b = *reinterpret_cast<const float2*>(bp + k * ldb);
        bv[0] = b.x; bv[1] = b.y;
      }
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (KS == 1) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) out(4 * mi + i, NJ * ni + j, acc[i][j]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float* pp = partial + (ks * M + 4 * mi + i) * Nc + NJ * ni;
        if constexpr (NJ == 4) *reinterpret_cast<float4*>(pp) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        else if constexpr (NJ == 3) { pp[0] = acc[i][0]; pp[1] = acc[i][1]; pp[2] = acc[i][2]; }
        else *reinterpret_cast<float2*>(pp) = make_float2(acc[i][0], acc[i][1]);
      }
    }
  }
  if (KS > 1) {
    bar();
    for (int w = t; w < M * Nc; w += nt) {
      float v = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) v += partial[ks * M * Nc + w];
      out(w / Nc, w % Nc, v);
    }
    bar();
  }
}

// The same over the whole block.
template <int KS, class Out>
__device__ __forceinline__ void block_gemm(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                                           int M, int Nc, int K, float* partial, Out out) {
  block_gemm_part<KS>(A, lda, B, ldb, M, Nc, K, partial, out, threadIdx.x, blockDim.x, [] { __syncthreads(); });
}

// ===========================================================================
// Predictor
// ===========================================================================
template <int N, bool TSM>
struct PredCfg : Dim<N> {
  using D = Dim<N>;
  static constexpr int TE = N >= 4 ? 8 : 16;
  static constexpr int THREADS = 256;
  static constexpr int CW = 12 * TE;                       // CK column width: (element, 9 fields + 3 pad)
  static constexpr int KS_SRC = N >= 4 ? 8 : 4;
  // shared memory carve-up (floats); tables only when TSM
  static constexpr int oVvT = 0;
  static constexpr int oVw = TSM ? round4(oVvT + D::L * D::NQP) : 0;
  static constexpr int oKtA = TSM ? round4(oVw + D::NQ * D::LP) : 0;
  // staged state rows, stride QSP: off the bank period, so that lanes on different
  // elements read different banks
  static constexpr int QSP = D::QS % 32 == 0 ? D::QS + 4 : D::QS;
  static constexpr int oQ = TSM ? round4(oKtA + 3 * D::L * D::LP) : 0;
  static constexpr int oC0 = oQ + TE * QSP;                // [L][8 TE] strains at t_n
  static constexpr int oR = oC0 + D::L * 8 * TE;           // [NQ][TE] damage rate at the nodes
  static constexpr int oP0 = round4(oR + D::NQ * TE);      // [L][CW] CK input
  static constexpr int oP1 = oP0 + D::L * CW;              // [L][CW] CK output
  static constexpr int oPart = oP1 + D::L * CW;            // split-K partial sums
  static constexpr int PART = KS_SRC * D::LP * TE;
  static constexpr int oCoef = oPart + PART;               // [TE][16]
  static constexpr int oGM = round4(oCoef + 16 * TE);      // [TE][40] GeomF, MatF as copied
  static constexpr int SMEM = oGM + 40 * TE;
  static constexpr bool FITS = SMEM * 4 <= 227 * 1024;
  static_assert(FITS || TSM, "predictor shared memory");
};

template <int N, bool TSM, int LAW>
__global__ void __launch_bounds__(256) k_predictor(StepArgs a) {
  using C = PredCfg<N, TSM>;
  constexpr int L = C::L, NQ = C::NQ, NQP = C::NQP, LP = C::LP, QS = C::QS, DS = C::DS, TE = C::TE;
  constexpr int CW = C::CW;
  constexpr TableLayout T = table_layout(N);
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const float* sVvT = TSM ? sm + C::oVvT : a.tables + T.VvT;
  const float* sVw = TSM ? sm + C::oVw : a.tables + T.Vw;
  const float* sKtA = TSM ? sm + C::oKtA : a.tables + T.KtA;
  float* sQ = sm + C::oQ;
  float* sC0 = sm + C::oC0;
  float* sR = sm + C::oR;
  float* sP0 = sm + C::oP0;
  float* sP1 = sm + C::oP1;
  float* sPart = sm + C::oPart;
  float* sCoef = sm + C::oCoef;
  float* sGM = sm + C::oGM;
  if (TSM) {
    copy_to_smem(sm + C::oVvT, a.tables + T.VvT, L * NQP);
    copy_to_smem(sm + C::oVw, a.tables + T.Vw, NQ * LP);
    copy_to_smem(sm + C::oKtA, a.tables + T.KtA, 3 * L * LP);
  }

  const int64_t ntiles = (a.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));
    __syncthreads();
    // one batch of asynchronous copies: the tile's state rows, GeomF and MatF
    for (int w = threadIdx.x; w < TE * QS / 4; w += blockDim.x) {
      const int e = w / (QS / 4), c = w - e * (QS / 4);
      if (e < ne) tc::cp_async16(sQ + e * C::QSP + 4 * c, a.q_in + (e0 + e) * QS + 4 * c);
      else *reinterpret_cast<float4*>(sQ + e * C::QSP + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int w = threadIdx.x; w < ne * 10; w += blockDim.x) {
      const int e = w / 10, k = w - 10 * e;
      if (k < 8) tc::cp_async16(sGM + e * 40 + 4 * k, reinterpret_cast<const float*>(a.geom + e0 + e) + 4 * k);
      else tc::cp_async16(sGM + e * 40 + 32 + 4 * (k - 8), reinterpret_cast<const float*>(a.mat + e0 + e) + 4 * (k - 8));
    }
    tc::cp_async_wait_all();
    __syncthreads();
    // per element: effective moduli at the cell mean (Eq. "effective-cdb", mu sign from Eq. "cdb-model")
    if (threadIdx.x < ne) {
      const int e = threadIdx.x;
      const int64_t ge = e0 + e;
      const MatF m = *reinterpret_cast<const MatF*>(sGM + e * 40 + 32);
      float lam, mu;
      effective_lame<LAW>(a.law, sQ + e * C::QSP, m, &lam, &mu);
      if (!(mu > 0.f) || !(lam + 2.f * mu > 0.f)) atomicOr(a.status, kStatusNonHyperbolic);
      a.cp[ge] = sqrtf(fmaxf(lam + 2.f * mu, 0.f) * m.rho_inv);
      float* c = sCoef + e * 16;
      c[0] = lam * m.rho_inv;
      c[1] = mu * m.rho_inv;
      const float* g = sGM + e * 40;           // GeomF starts with Theta^{-1}
      for (int k = 0; k < 9; ++k) c[2 + k] = g[k];
    }
    // coefficient arrays: strains at t_n [l][e*8 + c] and the CK input [l][e*12 + p]
    for (int w = threadIdx.x; w < L * TE; w += blockDim.x) {
      const int l = w / TE, e = w - l * TE;
      const float2* q2 = reinterpret_cast<const float2*>(sQ + e * C::QSP + l * 10);
      const float2 q01 = q2[0], q23 = q2[1], q45 = q2[2], q67 = q2[3], q89 = q2[4];
      float4* c0 = reinterpret_cast<float4*>(sC0 + l * 8 * TE + e * 8);
      float4* p0 = reinterpret_cast<float4*>(sP0 + l * CW + e * 12);
      c0[0] = make_float4(q01.x, q01.y, q23.x, q23.y);
      c0[1] = make_float4(q45.x, q45.y, q89.y, 0.f);
      p0[0] = make_float4(q01.x, q01.y, q23.x, q23.y);
      p0[1] = make_float4(q45.x, q45.y, q67.x, q67.y);
      p0[2] = make_float4(q89.x, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    // damage rate at the volume nodes from the state at t_n (two nodes per item)
    constexpr int NPAIR = NQP / 2;
    for (int w = threadIdx.x; w < TE * NPAIR; w += blockDim.x) {
      const int e = w / NPAIR, j = w - e * NPAIR;
      constexpr int NC = 7;                  // six strains and alpha at the node
      float acc[2][NC];
#pragma unroll
      for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int p = 0; p < NC; ++p) acc[n][p] = 0.f;
#pragma unroll 5
      for (int l = 0; l < L; ++l) {
        const float2 ph = *reinterpret_cast<const float2*>(sVvT + l * NQP + 2 * j);
        const float4 c0 = *reinterpret_cast<const float4*>(sC0 + l * 8 * TE + e * 8);
        const float4 c1 = *reinterpret_cast<const float4*>(sC0 + l * 8 * TE + e * 8 + 4);
        const float cv[NC] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z};
#pragma unroll
        for (int p = 0; p < NC; ++p) {
          acc[0][p] = fmaf(ph.x, cv[p], acc[0][p]);
          acc[1][p] = fmaf(ph.y, cv[p], acc[1][p]);
        }
      }
      const MatF m = *reinterpret_cast<const MatF*>(sGM + (e < ne ? e : 0) * 40 + 32);
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const int q = 2 * j + n;
        if (q < NQ) sR[q * TE + e] = e < ne ? law_rate<LAW>(a.law, acc[n], acc[n][6], m) : 0.f;
      }
    }
    __syncthreads();
    // D^1 of alpha = projection of the rate (mass matrix = identity)
    block_gemm<C::KS_SRC>(sVw, LP, sR, TE, LP, TE, NQ, sPart, [&](int k, int e, float v) {
      if (k < L && e < ne) a.d[(e0 + e) * DS + C::AOFF + k] = v;
    });

    // Cauchy-Kovalevskaya: D^i_kp = -sum_e Kt^e_kl D^{i-1}_lq (Theta^{-1}_ed B^d_pq); the
    // order loop is unrolled so that the mode counts are constants and the inner loop
    // can be software-pipelined
#pragma unroll
    for (int i = 1; i <= N; ++i) {
      const int Lin = n_modes(N - i + 1), Lout = n_modes(N - i);
      const float* pin = (i & 1) ? sP0 : sP1;
      float* pout = (i & 1) ? sP1 : sP0;
      const int doff = d_offset(N, i);
      for (int w = threadIdx.x; w < TE * Lout; w += blockDim.x) {
        const int k = w / TE, e = w - k * TE;
        float g[3][9];
#pragma unroll
        for (int f = 0; f < 9; ++f) g[0][f] = g[1][f] = g[2][f] = 0.f;
#pragma unroll 4
        for (int l = 0; l < Lin; ++l) {
          const float k0 = sKtA[(0 * L + l) * LP + k], k1 = sKtA[(1 * L + l) * LP + k], k2 = sKtA[(2 * L + l) * LP + k];
          const float4 p0 = *reinterpret_cast<const float4*>(pin + l * CW + e * 12);
          const float4 p1 = *reinterpret_cast<const float4*>(pin + l * CW + e * 12 + 4);
          const float p8 = pin[l * CW + e * 12 + 8];
          const float pv[9] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p8};
#pragma unroll
          for (int f = 0; f < 9; ++f) {
            g[0][f] = fmaf(k0, pv[f], g[0][f]);
            g[1][f] = fmaf(k1, pv[f], g[1][f]);
            g[2][f] = fmaf(k2, pv[f], g[2][f]);
          }
        }
        const float* c = sCoef + e * 16;
        float gd[3][9];   // d/dx_d of field f, projected
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int f = 0; f < 9; ++f) gd[d][f] = c[2 + d] * g[0][f] + c[5 + d] * g[1][f] + c[8 + d] * g[2][f];
        const float lr_ = c[0], mr = c[1];
        float Di[9];
        Di[0] = gd[0][6];
        Di[1] = gd[1][7];
        Di[2] = gd[2][8];
        Di[3] = 0.5f * (gd[1][6] + gd[0][7]);
        Di[4] = 0.5f * (gd[2][7] + gd[1][8]);
        Di[5] = 0.5f * (gd[0][8] + gd[2][6]);
        Di[6] = lr_ * (gd[0][0] + gd[0][1] + gd[0][2]) + 2.f * mr * (gd[0][0] + gd[1][3] + gd[2][5]);
        Di[7] = lr_ * (gd[1][0] + gd[1][1] + gd[1][2]) + 2.f * mr * (gd[0][3] + gd[1][1] + gd[2][4]);
        Di[8] = lr_ * (gd[2][0] + gd[2][1] + gd[2][2]) + 2.f * mr * (gd[0][5] + gd[1][4] + gd[2][2]);
        float* po = pout + k * CW + e * 12;
        *reinterpret_cast<float4*>(po) = make_float4(Di[0], Di[1], Di[2], Di[3]);
        *reinterpret_cast<float4*>(po + 4) = make_float4(Di[4], Di[5], Di[6], Di[7]);
        *reinterpret_cast<float4*>(po + 8) = make_float4(Di[8], 0.f, 0.f, 0.f);
        if (e < ne) {
          float* gout = a.d + (e0 + e) * DS + doff + k * 9;
#pragma unroll
          for (int f = 0; f < 9; ++f) gout[f] = Di[f];
        }
      }
      __syncthreads();
    }
  }
}

// ===========================================================================
// Predictor with the strains and alpha at the volume nodes on the tensor cores
// (degrees 2..4).  D[q][(e, c)] = sum_l phi_l(x_q) C_e[l][c], c = the six strains and
// alpha at t_n: 3xTF32 MMAs with A = phi_l(x_q) in tensor memory (lane q, column l,
// loaded once) and B = the tile's coefficients in shared memory (row (e, c), K = l),
// issued before the CK recursion, which runs on the SIMT cores meanwhile; then the
// damage rate at the nodes from D and its projection (D^1 of alpha).  Two CTAs of 256
// threads per SM, each with 256 tensor-memory columns.
// ===========================================================================
template <int N>
struct PredTcCfg : Dim<N> {
  using D = Dim<N>;
  static constexpr int TE = N >= 4 ? 8 : 16;
  static constexpr int THREADS = 256;
  static constexpr int CW = 12 * TE;                       // CK column width: (element, 9 fields + 3 pad)
  static constexpr int KS_SRC = N >= 4 ? 8 : 4;
  static constexpr int KP = tc_kp(N);
  static constexpr int NB = 8 * TE;                        // MMA N: (element, 6 strains, alpha, 0)
  // B's 8-row groups (one per element) BSBO floats apart: 4 floats off the bank period, so
  // that the lanes of a warp writing one coefficient of eight elements hit distinct banks
  static constexpr int BSBO = 8 * KP + 4;
  static constexpr int COL_D = 0, COL_AH = NB, COL_AL = NB + KP;
  static constexpr int TMEM_NEED = COL_AL + KP;
  static constexpr int TMEM_COLS = TMEM_NEED <= 128 ? 128 : 256;
  static constexpr int QSP = D::QS % 32 == 0 ? D::QS + 4 : D::QS;
  static constexpr int oVw = 0;                            // [NQ][LP]
  static constexpr int oKtA = round4(oVw + D::NQ * D::LP); // [L][LP][4]: Kt^e_lk of e = 0..2 (and 0) in one 16-byte word
  static constexpr int oQ = round4(oKtA + 4 * D::L * D::LP);   // [TE][QSP] staged state rows
  static constexpr int oBH = oQ + TE * QSP;                // B, TF32 high part
  static constexpr int oBL = oBH + TE * BSBO;              // B, remainder
  static constexpr int oR = oBL + TE * BSBO;               // [NQ][TE] damage rate at the nodes
  static constexpr int oP0 = round4(oR + D::NQ * TE);      // [L][CW] CK input
  static constexpr int oP1 = oP0 + D::L * CW;              // [L][CW] CK output
  static constexpr int oPart = oP1 + D::L * CW;            // split-K partial sums
  static constexpr int PART = KS_SRC * D::LP * TE;
  static constexpr int oCoef = oPart + PART;               // [TE][16]
  static constexpr int oGM = round4(oCoef + 16 * TE);      // [TE][40] GeomF, MatF as copied
  static constexpr int SMEM = oGM + 40 * TE;
  static constexpr int ISSUER = THREADS - 32;
  __host__ __device__ static constexpr int b_index(int e, int c, int l) {
    return e * BSBO + (l >> 2) * 32 + c * 4 + (l & 3);
  }
  static_assert(NB % 16 == 0 && NB <= 256 && D::NQ <= 128 && KP % 8 == 0 && KP <= 40, "tensor-core shapes");
  static_assert(oQ % 4 == 0 && (TE * QSP) % 4 == 0 && BSBO % 4 == 0, "16-byte aligned operands");
  static_assert(TMEM_NEED <= 256, "two CTAs per SM share the 512 tensor-memory columns");
  static_assert(2 * (SMEM * 4 + 1024) <= 228 * 1024, "two CTAs per SM");
  static_assert(TE % 8 == 0 && THREADS == 256, "read-out: warps 0-3 and 4-7 take half the elements each");
  static_assert(TE * n_modes(N - 1) <= ISSUER, "the issuing warp has no CK work at order 1");
};

template <int N, int LAW>
__global__ void __launch_bounds__(256, 2) k_predictor_tc(StepArgs a) {
  using C = PredTcCfg<N>;
  constexpr int L = C::L, NQ = C::NQ, LP = C::LP, QS = C::QS, DS = C::DS, TE = C::TE, KP = C::KP;
  constexpr int CW = C::CW, NB = C::NB;
  constexpr TableLayout T = table_layout(N);
  constexpr int kWaitLimit = 1 << 24;
  const int wait_limit = a.wait_limit_set ? a.wait_limit : kWaitLimit;
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const float* sVw = sm + C::oVw;
  const float* sKtA = sm + C::oKtA;
  float* sQ = sm + C::oQ;
  float* sBH = sm + C::oBH;
  float* sBL = sm + C::oBL;
  float* sR = sm + C::oR;
  float* sP0 = sm + C::oP0;
  float* sP1 = sm + C::oP1;
  float* sPart = sm + C::oPart;
  float* sCoef = sm + C::oCoef;
  float* sGM = sm + C::oGM;
  const float* tb = a.tables;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  copy_to_smem(sm + C::oVw, tb + T.Vw, NQ * LP);
  for (int w = tid; w < L * LP; w += blockDim.x) {
    const int l = w / LP, k = w - l * LP;
    *reinterpret_cast<float4*>(sm + C::oKtA + 4 * w) =
        make_float4(__ldg(tb + T.KtA + (0 * L + l) * LP + k), __ldg(tb + T.KtA + (1 * L + l) * LP + k),
                    __ldg(tb + T.KtA + (2 * L + l) * LP + k), 0.f);
  }
  // B's K padding (modes L .. KP-1) stays zero
  if constexpr (KP > L) {
    for (int w = tid; w < TE * 8 * (KP - L); w += blockDim.x) {
      const int l = L + w % (KP - L), ec = w / (KP - L);
      sBH[C::b_index(ec >> 3, ec & 7, l)] = 0.f;
      sBL[C::b_index(ec >> 3, ec & 7, l)] = 0.f;
    }
  }
  if (warp == 0) tc::alloc(&tmem_base, C::TMEM_COLS);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  // A = phi_l(x_q) (TF32 part, remainder) into tensor memory once: lane q, columns l, read
  // from the canonical tables (rows q >= NQ are zero)
  if (warp < 4) {
    const int q = 32 * warp + lane;
    const uint32_t lane_base = static_cast<uint32_t>(32 * warp) << 16;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const float* src = tb + (part ? T.PhiL : T.PhiH);
      float v[KP];
#pragma unroll
      for (int j = 0; j < KP / 4; ++j) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(src + tc_canon(q, 4 * j, KP)));
        v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
      }
      tc::st_cols<KP>(tmem + lane_base + (part ? C::COL_AL : C::COL_AH), v);
    }
    tc::wait_st();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  uint32_t phase = 0;
  bool failed = false;

  const int64_t ntiles = (a.E + TE - 1) / TE;
  // one batch of asynchronous copies of a tile: its state rows, GeomF and MatF (rows of
  // elements beyond the mesh are zero)
  auto issue = [&](int64_t tl) {
    const int64_t t0 = tl * TE;
    const int nt = static_cast<int>(min(static_cast<int64_t>(TE), a.E - t0));
    for (int w = tid; w < TE * QS / 4; w += blockDim.x) {
      const int e = w / (QS / 4), c = w - e * (QS / 4);
      if (e < nt) tc::cp_async16(sQ + e * C::QSP + 4 * c, a.q_in + (t0 + e) * QS + 4 * c);
      else *reinterpret_cast<float4*>(sQ + e * C::QSP + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int w = tid; w < nt * 10; w += blockDim.x) {
      const int e = w / 10, k = w - 10 * e;
      if (k < 8) tc::cp_async16(sGM + e * 40 + 4 * k, reinterpret_cast<const float*>(a.geom + t0 + e) + 4 * k);
      else tc::cp_async16(sGM + e * 40 + 32 + 4 * (k - 8), reinterpret_cast<const float*>(a.mat + t0 + e) + 4 * (k - 8));
    }
    tc::cp_async_commit();
  };
  if (static_cast<int64_t>(blockIdx.x) < ntiles) issue(blockIdx.x);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));
    tc::cp_async_wait<0>();                  // this tile's copies (issued during the previous tile's CK)
    __syncthreads();
    // per element: effective moduli at the cell mean (Eq. "effective-cdb", mu sign from Eq. "cdb-model")
    if (tid < ne) {
      const int e = tid;
      const int64_t ge = e0 + e;
      const MatF m = *reinterpret_cast<const MatF*>(sGM + e * 40 + 32);
      float lam, mu;
      effective_lame<LAW>(a.law, sQ + e * C::QSP, m, &lam, &mu);
      if (!(mu > 0.f) || !(lam + 2.f * mu > 0.f)) atomicOr(a.status, kStatusNonHyperbolic);
      a.cp[ge] = sqrtf(fmaxf(lam + 2.f * mu, 0.f) * m.rho_inv);
      float* c = sCoef + e * 16;
      c[0] = lam * m.rho_inv;
      c[1] = mu * m.rho_inv;
      const float* g = sGM + e * 40;           // GeomF starts with Theta^{-1}
      for (int k = 0; k < 9; ++k) c[2 + k] = g[k];
      // what the damage rate at the nodes needs of the material (GeomF and MatF are
      // overwritten by the next tile's copies meanwhile)
      c[11] = m.lam0;
      c[12] = m.mu0;
      c[13] = m.gamma_r;
      c[14] = m.xi0;
      c[15] = m.cd;
    }
    // the MMA's B operand (strains and alpha at t_n, split) and the CK input [l][e*12 + p]
    for (int w = tid; w < L * TE; w += blockDim.x) {
      const int l = w / TE, e = w - l * TE;
      const float2* q2 = reinterpret_cast<const float2*>(sQ + e * C::QSP + l * 10);
      const float2 q01 = q2[0], q23 = q2[1], q45 = q2[2], q67 = q2[3], q89 = q2[4];
      const float x[8] = {q01.x, q01.y, q23.x, q23.y, q45.x, q45.y, q89.y, 0.f};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float h = tc::tf32_hi(x[c]);
        sBH[C::b_index(e, c, l)] = h;
        sBL[C::b_index(e, c, l)] = tc::tf32_hi(x[c] - h);
      }
      float4* p0 = reinterpret_cast<float4*>(sP0 + l * CW + e * 12);
      p0[0] = make_float4(q01.x, q01.y, q23.x, q23.y);
      p0[1] = make_float4(q45.x, q45.y, q67.x, q67.y);
      p0[2] = make_float4(q89.x, 0.f, 0.f, 0.f);
    }
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncthreads();
    // the next tile's copies: the state rows, GeomF and MatF are no longer read
    if (tile + gridDim.x < ntiles) issue(tile + gridDim.x);
    // issued from the last warp, which has no CK work at order 1 (the issuing thread waits
    // for the tensor pipe)
    if (tid == C::ISSUER) {
      tc::fence_after();
      constexpr uint32_t idesc = tc::idesc_tf32(128, NB);
      const uint32_t bH = tc::smem_u32(sBH), bL = tc::smem_u32(sBL);
      constexpr uint32_t sbo = 4u * C::BSBO;
#pragma unroll
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint32_t off = ks * 256;   // 8 K-elements = 2 core matrices
        const uint32_t aH = tmem + C::COL_AH + 8 * ks, aL = tmem + C::COL_AL + 8 * ks;
        tc::mma_tf32_ta(tmem + C::COL_D, aH, tc::desc_kmajor_strided(bH + off, 128u, sbo), idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ta(tmem + C::COL_D, aH, tc::desc_kmajor_strided(bL + off, 128u, sbo), idesc, 1u);
        tc::mma_tf32_ta(tmem + C::COL_D, aL, tc::desc_kmajor_strided(bH + off, 128u, sbo), idesc, 1u);
      }
      tc::commit(&mbar);
    }

    // Cauchy-Kovalevskaya while the MMAs run: D^i_kp = -sum_e Kt^e_kl D^{i-1}_lq
    // (Theta^{-1}_ed B^d_pq); the order loop is unrolled so that the mode counts are constants
#pragma unroll
    for (int i = 1; i <= N; ++i) {
      const int Lin = n_modes(N - i + 1), Lout = n_modes(N - i);
      const float* pin = (i & 1) ? sP0 : sP1;
      float* pout = (i & 1) ? sP1 : sP0;
      const int doff = d_offset(N, i);
      for (int w = tid; w < TE * Lout; w += blockDim.x) {
        const int k = w / TE, e = w - k * TE;
        float g[3][9];
#pragma unroll
        for (int f = 0; f < 9; ++f) g[0][f] = g[1][f] = g[2][f] = 0.f;
#pragma unroll 4
        for (int l = 0; l < Lin; ++l) {
          const float4 kk = *reinterpret_cast<const float4*>(sKtA + 4 * (l * LP + k));
          const float k0 = kk.x, k1 = kk.y, k2 = kk.z;
          const float4 p0 = *reinterpret_cast<const float4*>(pin + l * CW + e * 12);
          const float4 p1 = *reinterpret_cast<const float4*>(pin + l * CW + e * 12 + 4);
          const float p8 = pin[l * CW + e * 12 + 8];
          const float pv[9] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p8};
#pragma unroll
          for (int f = 0; f < 9; ++f) {
            g[0][f] = fmaf(k0, pv[f], g[0][f]);
            g[1][f] = fmaf(k1, pv[f], g[1][f]);
            g[2][f] = fmaf(k2, pv[f], g[2][f]);
          }
        }
        const float* c = sCoef + e * 16;
        float gd[3][9];   // d/dx_d of field f, projected
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int f = 0; f < 9; ++f) gd[d][f] = c[2 + d] * g[0][f] + c[5 + d] * g[1][f] + c[8 + d] * g[2][f];
        const float lr_ = c[0], mr = c[1];
        float Di[9];
        Di[0] = gd[0][6];
        Di[1] = gd[1][7];
        Di[2] = gd[2][8];
        Di[3] = 0.5f * (gd[1][6] + gd[0][7]);
        Di[4] = 0.5f * (gd[2][7] + gd[1][8]);
        Di[5] = 0.5f * (gd[0][8] + gd[2][6]);
        Di[6] = lr_ * (gd[0][0] + gd[0][1] + gd[0][2]) + 2.f * mr * (gd[0][0] + gd[1][3] + gd[2][5]);
        Di[7] = lr_ * (gd[1][0] + gd[1][1] + gd[1][2]) + 2.f * mr * (gd[0][3] + gd[1][1] + gd[2][4]);
        Di[8] = lr_ * (gd[2][0] + gd[2][1] + gd[2][2]) + 2.f * mr * (gd[0][5] + gd[1][4] + gd[2][2]);
        float* po = pout + k * CW + e * 12;
        *reinterpret_cast<float4*>(po) = make_float4(Di[0], Di[1], Di[2], Di[3]);
        *reinterpret_cast<float4*>(po + 4) = make_float4(Di[4], Di[5], Di[6], Di[7]);
        *reinterpret_cast<float4*>(po + 8) = make_float4(Di[8], 0.f, 0.f, 0.f);
        if (e < ne) {
          float* gout = a.d + (e0 + e) * DS + doff + k * 9;
#pragma unroll
          for (int f = 0; f < 9; ++f) gout[f] = Di[f];
        }
      }
      __syncthreads();
    }

    // damage rate at the volume nodes from the MMA's result: thread (warp w, lane) holds
    // node q = 32 (w mod 4) + lane of elements [TE/2 (w / 4), TE/2 (w / 4 + 1))
    const bool ok = tc::wait_parity(&mbar, phase, wait_limit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after();
    {
      const int q = 32 * (warp & 3) + lane;
      const uint32_t lane_base = static_cast<uint32_t>(32 * (warp & 3)) << 16;
#pragma unroll 1
      for (int e4 = 0; e4 < TE / 2; e4 += 4) {
        const int eb = (warp >> 2) * (TE / 2) + e4;
        float v[32];
        tc::ld_cols<32>(tmem + lane_base + C::COL_D + 8 * eb, v);
        tc::wait_ld();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int e = eb + j;
          const float* c = sCoef + (e < ne ? e : 0) * 16;
          MatF m{};
          m.lam0 = c[11]; m.mu0 = c[12]; m.gamma_r = c[13]; m.xi0 = c[14]; m.cd = c[15];
          if (q < NQ) sR[q * TE + e] = e < ne ? law_rate<LAW>(a.law, v + 8 * j, v[8 * j + 6], m) : 0.f;
        }
      }
    }
    tc::fence_before();
    __syncthreads();
    // D^1 of alpha = projection of the rate (mass matrix = identity)
    block_gemm<C::KS_SRC>(sVw, LP, sR, TE, LP, TE, NQ, sPart, [&](int k, int e, float v) {
      if (k < L && e < ne) a.d[(e0 + e) * DS + C::AOFF + k] = v;
    });
  }
  tc::cp_async_wait<0>();                    // no copy may still be in flight at exit
  if (failed) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    tc::wait_parity(&mbar, phase ^ 1u, kWaitLimit);   // let the MMAs in flight finish before freeing TMEM
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, C::TMEM_COLS);
}

// ===========================================================================
// Picard predictor (the extension Sec. 5.1 proposes in place of the linearised
// CK): starting from the CK output in a.d, each iteration evaluates the
// element-local rate R(q) = -div F(q) + S(q) of the predictor's polynomial
// q(t) = sum_o t^o/o! D^o at the N + 1 time nodes of the step, with the volume-
// rule projection of Theta^{-1} F(q) and of the damage rate and the divergence
// through the Kt tables, and replaces D^{j+1} by the j-th Taylor coefficient of
// the polynomial through those values.  Each D^o keeps the CK's form (degree
// N - o for the wave fields, D^1 only for alpha).  Persistent CTAs of 512 threads,
// TE elements per tile, all iterations in shared memory; everything SIMT.
// ===========================================================================
template <int N>
struct PicardCfg : Dim<N> {
  using D = Dim<N>;
  static constexpr int TE = 4;
  static constexpr int THREADS = 512;
  static constexpr int CU = TE * 12;                       // node-value columns: (element, 10 fields + 2 pad)
  static constexpr int CF = TE * 28;                       // flux columns: (element, e' 0..2 x 9 fields, rate)
  static constexpr int FST = CF + 4;                       // row stride of the nodal fluxes
  static constexpr int QSP = D::QS % 32 == 0 ? D::QS + 4 : D::QS;
  static constexpr int VQ = round4(D::NQ);                 // volume nodes padded to a multiple of 4
  static constexpr int oVvT = 0;                           // [L][VQ] phi_l(x_q), zero beyond NQ
  static constexpr int oVw = round4(oVvT + D::L * VQ);     // [NQ][LP]
  static constexpr int oKtA = round4(oVw + D::NQ * D::LP); // [3][L][LP]
  static constexpr int oQ = round4(oKtA + 3 * D::L * D::LP);   // [TE][QSP] state at t_n
  static constexpr int oD = oQ + TE * QSP;                 // [TE][DS] Taylor coefficients being refined
  static constexpr int oGeo = round4(oD + TE * D::DS);     // [TE][40] GeomF, MatF as copied
  static constexpr int oUt = oGeo + TE * 40;               // [L][CU] modal values at one time node
  static constexpr int oU = round4(oUt + D::L * CU);       // [VQ][CU] node values; later [LP][CF] projections
  static constexpr int U_SIZE = (VQ * CU > D::LP * CF ? VQ * CU : D::LP * CF);
  static constexpr int oF = round4(oU + U_SIZE);           // [VQ][FST] nodal reference fluxes and rate
  static constexpr int oDn = oF + VQ * FST;                // [TE][DS] new coefficients (same layout as oD)
  static constexpr int oTc = oDn + TE * D::DS;             // [NT][N+1] t_z^o / o!, then [NT][NT] the fit
  static constexpr int SMEM = round4(oTc + D::NT * (N + 1) + D::NT * D::NT);
  static constexpr bool FITS = SMEM * 4 <= 227 * 1024;    // N = 5 does not fit
  static_assert(D::LP % 4 == 0 && CU % 4 == 0 && CF % 4 == 0 && FST % 4 == 0, "block GEMM shapes");
};

template <int N, int LAW>
__global__ void __launch_bounds__(512, 1) k_picard(StepArgs a) {
  using C = PicardCfg<N>;
  constexpr int L = C::L, NQ = C::NQ, NQP = C::NQP, LP = C::LP, NT = C::NT, QS = C::QS, DS = C::DS;
  constexpr int AOFF = C::AOFF, TE = C::TE, CU = C::CU, CF = C::CF, FST = C::FST, QSP = C::QSP, VQ = C::VQ;
  constexpr int L1 = n_modes(N - 1);
  constexpr TableLayout T = table_layout(N);
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* sVvT = sm + C::oVvT;
  float* sVw = sm + C::oVw;
  float* sKtA = sm + C::oKtA;
  float* sQ = sm + C::oQ;
  float* sD = sm + C::oD;
  float* sGM = sm + C::oGeo;
  float* sUt = sm + C::oUt;
  float* sU = sm + C::oU;
  float* sFh = sm + C::oU;                                 // the projections reuse the node-value rows
  float* sF = sm + C::oF;
  float* sDn = sm + C::oDn;
  float* sCz = sm + C::oTc;                                // [NT][N+1]
  float* sFit = sCz + NT * (N + 1);                        // [NT][NT], sFit[j][z]
  const float* tb = a.tables;
  const float dt = a.dt;
  for (int w = threadIdx.x; w < L * VQ; w += blockDim.x) {
    const int l = w / VQ, q = w - l * VQ;
    sVvT[w] = q < NQ ? __ldg(tb + T.VvT + l * NQP + q) : 0.f;
  }
  copy_to_smem(sVw, tb + T.Vw, NQ * LP);
  copy_to_smem(sKtA, tb + T.KtA, 3 * L * LP);
  // Taylor weights t_z^o / o! and the fit Tfit[j][z] / dt^j
  if (threadIdx.x < NT) {
    const int z = threadIdx.x;
    const float tz = __ldg(tb + T.tz + z) * dt;
    float c = 1.f;
    for (int o = 0; o <= N; ++o) {
      sCz[z * (N + 1) + o] = c;
      c *= tz / static_cast<float>(o + 1);
    }
    float sc = 1.f;
    for (int j = 0; j < NT; ++j) {
      for (int zz = 0; zz < NT; ++zz) {
        if (zz == z) sFit[j * NT + zz] = __ldg(tb + T.Tfit + j * NT + zz) * sc;
      }
      sc /= dt;
    }
  }

  const int64_t ntiles = (a.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));
    __syncthreads();
    for (int w = threadIdx.x; w < TE * QS / 4; w += blockDim.x) {
      const int e = w / (QS / 4), c = w - e * (QS / 4);
      if (e < ne) tc::cp_async16(sQ + e * QSP + 4 * c, a.q_in + (e0 + e) * QS + 4 * c);
      else *reinterpret_cast<float4*>(sQ + e * QSP + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int w = threadIdx.x; w < TE * DS / 4; w += blockDim.x) {
      const int e = w / (DS / 4), c = w - e * (DS / 4);
      if (e < ne) tc::cp_async16(sD + e * DS + 4 * c, a.d + (e0 + e) * DS + 4 * c);
      else *reinterpret_cast<float4*>(sD + e * DS + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int w = threadIdx.x; w < ne * 10; w += blockDim.x) {
      const int e = w / 10, k = w - 10 * e;
      if (k < 8) tc::cp_async16(sGM + e * 40 + 4 * k, reinterpret_cast<const float*>(a.geom + e0 + e) + 4 * k);
      else tc::cp_async16(sGM + e * 40 + 32 + 4 * (k - 8), reinterpret_cast<const float*>(a.mat + e0 + e) + 4 * (k - 8));
    }
    tc::cp_async_wait_all();
    __syncthreads();

#pragma unroll 1
    for (int iter = 0; iter < a.picard_iters; ++iter) {
      for (int w = threadIdx.x; w < TE * DS; w += blockDim.x) sDn[w] = 0.f;
#pragma unroll 1
      for (int z = 0; z < NT; ++z) {
        // modal values of q(t_z): (element, field) columns; alpha to first order
        for (int w = threadIdx.x; w < L * TE; w += blockDim.x) {
          const int l = w / TE, e = w - l * TE;
          const float* q = sQ + e * QSP + l * 10;
          const float* de = sD + e * DS;
          float u[12];
#pragma unroll
          for (int c = 0; c < 10; ++c) u[c] = q[c];
          u[10] = u[11] = 0.f;
#pragma unroll
          for (int o = 1; o <= N; ++o) {
            if (l < n_modes(N - o)) {
#pragma unroll
              for (int c = 0; c < 9; ++c) u[c] = fmaf(sCz[z * (N + 1) + o], de[d_offset(N, o) + l * 9 + c], u[c]);
            }
          }
          u[9] = fmaf(sCz[z * (N + 1) + 1], de[AOFF + l], u[9]);
          float4* dst = reinterpret_cast<float4*>(sUt + l * CU + e * 12);
          dst[0] = make_float4(u[0], u[1], u[2], u[3]);
          dst[1] = make_float4(u[4], u[5], u[6], u[7]);
          dst[2] = make_float4(u[8], u[9], 0.f, 0.f);
        }
        __syncthreads();
        // node values U[q][col] = sum_l phi_l(x_q) Ut[l][col]
        block_gemm<1>(sVvT, VQ, sUt, CU, VQ, CU, L, nullptr, [&](int q, int col, float v) { sU[q * CU + col] = v; });
        __syncthreads();
        // reference fluxes Theta^{-1}_{e'd} F^d and the damage rate at every node
        for (int w = threadIdx.x; w < NQ * TE; w += blockDim.x) {
          const int q = w / TE, e = w - q * TE;
          float* f = sF + q * FST + e * 28;
          if (e >= ne) {
#pragma unroll
            for (int p = 0; p < 28; ++p) f[p] = 0.f;
            continue;
          }
          const float* u = sU + q * CU + e * 12;
          const float* gm = sGM + e * 40;
          const MatF m = *reinterpret_cast<const MatF*>(gm + 32);
          float sig[6], r;
          law_point<LAW>(a.law, u, u[9], m, sig, &r);
          const float S[3][3] = {{sig[0], sig[3], sig[5]}, {sig[3], sig[1], sig[4]}, {sig[5], sig[4], sig[2]}};
          const float v[3] = {u[6], u[7], u[8]};
#pragma unroll
          for (int ep = 0; ep < 3; ++ep) {
            const float th[3] = {gm[ep * 3 + 0], gm[ep * 3 + 1], gm[ep * 3 + 2]};   // Theta^{-1}[e'][d]
            float* fe = f + ep * 9;
            // strain rows: -(v_i th_j + v_j th_i) / 2 ; velocity rows: -(sigma th)_i / rho
            fe[0] = -v[0] * th[0];
            fe[1] = -v[1] * th[1];
            fe[2] = -v[2] * th[2];
            fe[3] = -0.5f * (v[0] * th[1] + v[1] * th[0]);
            fe[4] = -0.5f * (v[1] * th[2] + v[2] * th[1]);
            fe[5] = -0.5f * (v[2] * th[0] + v[0] * th[2]);
#pragma unroll
            for (int i = 0; i < 3; ++i) fe[6 + i] = -m.rho_inv * (S[i][0] * th[0] + S[i][1] * th[1] + S[i][2] * th[2]);
          }
          f[27] = r;
        }
        __syncthreads();
        // projections by the volume rule: Fh[l][col] = sum_q w_q phi_l(x_q) F[q][col]
        // 4 x 2 work items: (LP/4) x (CF/2) of them fill the block
        block_gemm_part<1, 2>(sVw, LP, sF, FST, LP, CF, NQ, nullptr, [&](int l, int col, float v) { sFh[l * CF + col] = v; },
                              threadIdx.x, blockDim.x, [] { __syncthreads(); });
        __syncthreads();
        // R(t_z) = -sum_e' Kt^{e'} Fh_{e'} + Shat, folded into the Taylor fit of every order
        // items (mode, element, group of 3 fields)
        for (int w = threadIdx.x; w < L * TE * 3; w += blockDim.x) {
          const int pg = w % 3, ke = w / 3;
          const int k = ke / TE, e = ke - k * TE;
          float* dn = sDn + e * DS;
          if (k < L1) {
            float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll 5
            for (int l = 0; l < L; ++l) {
              const float* fh = sFh + l * CF + e * 28 + 3 * pg;
#pragma unroll
              for (int ep = 0; ep < 3; ++ep) {
                const float kt = sKtA[(ep * L + l) * LP + k];
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[j] = fmaf(kt, fh[ep * 9 + j], acc[j]);
              }
            }
#pragma unroll
            for (int o = 1; o <= N; ++o) {
              if (k < n_modes(N - o)) {
#pragma unroll
                for (int j = 0; j < 3; ++j) dn[d_offset(N, o) + k * 9 + 3 * pg + j] -= sFit[(o - 1) * NT + z] * acc[j];
              }
            }
          }
          if (pg == 0) dn[AOFF + k] += sFit[z] * sFh[k * CF + e * 28 + 27];
        }
        __syncthreads();
      }
      for (int w = threadIdx.x; w < TE * DS; w += blockDim.x) sD[w] = sDn[w];
      __syncthreads();
    }
    bool bad = false;
    for (int w = threadIdx.x; w < ne * DS; w += blockDim.x) {
      bad |= !isfinite(sD[w]);
      a.d[e0 * DS + w] = sD[w];
    }
    if (bad) atomicOr(a.status, kStatusNonFinite);
  }
}

// ===========================================================================
// Picard predictor with its two contractions on the tensor cores (degrees 2..4).
// Per time node t_z of an iteration: the node values of the predictor's
// polynomial, U[q][(e, c)] = sum_l phi_l(x_q) q_l(t_z) (A = phi_l(x_q) in tensor
// memory, lane = node; B = the modal values at t_z, columns (element, field)),
// and the projection of the nodal reference fluxes Theta^{-1}_{e'd} F^d and the
// damage rate, Fh[l][(e, e' x field | rate)] = sum_q w_q phi_l(x_q) F[q][.]
// (A = w_q phi_l(x_q) in tensor memory, lane = mode; B = the nodal terms), both
// in 3xTF32 as in the corrector.  The pointwise flux reads the node values
// straight from tensor memory; the divergence through the Kt tables and the time
// fit stay SIMT.  Four elements per tile (one warp group each in the flux phase),
// 512 threads, one CTA per SM; the last warp issues the MMAs.
// ===========================================================================
template <int N>
struct PicTcCfg : Dim<N> {
  using D = Dim<N>;
  static constexpr int TE = 4;
  static constexpr int THREADS = 512;
  static constexpr int KP = tc_kp(N), KQ = tc_kq(N);
  static constexpr int NU = (TE * 12 + 15) / 16 * 16;      // node-value MMA N: (element, 12 channels), padded
  static constexpr int CF = TE * 28;                       // nodal-term columns (element, e' x 9 fields, rate)
  static constexpr int NPF = (CF + 15) / 16 * 16;          // projection MMA N
  // the projection's B operand: core matrices 36 floats apart along K, so that the 32
  // nodes one warp writes land in 32 banks
  static constexpr int PLBO = 36, PGS = KQ / 4 * PLBO, BF = NPF / 8 * PGS;
  static constexpr int COL_U = 0;                          // node values: lane q, NU columns
  static constexpr int COL_F = NU;                         // projections: lane l, NPF columns
  static constexpr int COL_AH = COL_F + NPF, COL_AL = COL_AH + KQ;   // projection A (w phi), lane = mode
  static constexpr int COL_PH = COL_AL + KQ, COL_PL = COL_PH + KP;   // node-value A (phi), lane = node
  static constexpr int TMEM_NEED = COL_PL + KP;
  static constexpr int TMEM_COLS = TMEM_NEED <= 128 ? 128 : (TMEM_NEED <= 256 ? 256 : 512);
  static constexpr int QSP = D::QS % 32 == 0 ? D::QS + 4 : D::QS;
  static constexpr int oKtA = 0;                                       // [3][L][LP]
  static constexpr int oQ = round4(oKtA + 3 * D::L * D::LP);           // [TE][QSP] state at t_n
  static constexpr int oD = oQ + TE * QSP;                             // [TE][DS] coefficients being refined
  static constexpr int oDn = oD + TE * D::DS;                          // [TE][DS] new coefficients
  static constexpr int oGeo = round4(oDn + TE * D::DS);                // [TE][40] GeomF, MatF
  static constexpr int oBuH = round4(oGeo + TE * 40);                  // [NU x KP] canonical K-major
  static constexpr int oBuL = oBuH + NU * KP;
  static constexpr int oBfH = oBuL + NU * KP;                          // [NPF x KQ] padded K-major
  static constexpr int oBfL = oBfH + BF;
  static constexpr int oFh = oBfL + BF;                                // [LP][CF] projections
  static constexpr int oC = oFh + D::LP * CF;                          // [CF] nodal terms at node 0
  static constexpr int oTc = round4(oC + CF);                          // [NT][N+1] t_z^o / o!, [NT][NT] fit
  static constexpr int SMEM = round4(oTc + D::NT * (N + 1) + D::NT * D::NT);
  static constexpr int ISSUER = THREADS - 32;
  static_assert(D::NQ <= 128 && KQ <= 128 && KP <= 40 && TMEM_NEED <= 512, "tensor-core shapes");
  static_assert(TE * 12 <= NU && NU % 16 == 0 && NPF % 16 == 0 && NPF <= 256 && CF % 16 == 0, "MMA N and read-out");
  static_assert(4 * TE <= THREADS / 32, "one warp group per element in the flux phase");
  static_assert(SMEM * 4 <= 227 * 1024, "Picard tensor-core shared memory");
  __host__ __device__ static constexpr int prj_canon(int n, int q) {
    return (n >> 3) * PGS + (q >> 2) * PLBO + (n & 7) * 4 + (q & 3);
  }
};

template <int N, int LAW>
__global__ void __launch_bounds__(PicTcCfg<N>::THREADS, 1) k_picard_tc(StepArgs a) {
  using C = PicTcCfg<N>;
  constexpr int L = C::L, NQ = C::NQ, LP = C::LP, NT = C::NT, QS = C::QS, DS = C::DS, AOFF = C::AOFF;
  constexpr int TE = C::TE, KP = C::KP, KQ = C::KQ, NU = C::NU, CF = C::CF, NPF = C::NPF, QSP = C::QSP;
  constexpr int L1 = n_modes(N - 1);
  constexpr TableLayout T = table_layout(N);
  constexpr int kWaitLimit = 1 << 24;
  const int wait_limit = a.wait_limit_set ? a.wait_limit : kWaitLimit;
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  float* sKtA = sm + C::oKtA;
  float* sQ = sm + C::oQ;
  float* sD = sm + C::oD;
  float* sDn = sm + C::oDn;
  float* sGM = sm + C::oGeo;
  float* sBuH = sm + C::oBuH;
  float* sBuL = sm + C::oBuL;
  float* sBfH = sm + C::oBfH;
  float* sBfL = sm + C::oBfL;
  float* sFh = sm + C::oFh;
  float* sC = sm + C::oC;
  float* sCz = sm + C::oTc;                                // [NT][N+1]
  float* sFit = sCz + NT * (N + 1);                        // [NT][NT], sFit[j][z]
  const float* tb = a.tables;
  const float dt = a.dt;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  copy_to_smem(sKtA, tb + T.KtA, 3 * L * LP);
  for (int w = tid; w < 2 * C::BF; w += blockDim.x) sBfH[w] = 0.f;   // rows beyond CF stay zero
  if (tid < NT) {
    const int z = tid;
    const float tz = __ldg(tb + T.tz + z) * dt;
    float c = 1.f;
    for (int o = 0; o <= N; ++o) {
      sCz[z * (N + 1) + o] = c;
      c *= tz / static_cast<float>(o + 1);
    }
    float sc = 1.f;
    for (int j = 0; j < NT; ++j) {
      sFit[j * NT + z] = __ldg(tb + T.Tfit + j * NT + z) * sc;
      sc /= dt;
    }
  }
  if (warp == 0) tc::alloc(&tmem_base, C::TMEM_COLS);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  // constant A operands into tensor memory: w_q phi_l(x_q) (lane l, columns q) on warps 0-3,
  // phi_l(x_q) (lane q, columns l) on warps 4-7, TF32 parts and remainders
  if (warp < 4) {
    const uint32_t lane_base = static_cast<uint32_t>(32 * warp) << 16;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const float* src = tb + (part ? T.PrjL : T.PrjH) + (32 * warp + lane) * KQ;
#pragma unroll 1
      for (int c0 = 0; c0 < KQ; c0 += 32) {
        float v[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 x = __ldg(reinterpret_cast<const float4*>(src + c0) + j);
          v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
        }
        tc::st_x32(tmem + lane_base + (part ? C::COL_AL : C::COL_AH) + c0, v);
      }
    }
  } else if (warp < 8) {
    const int q = 32 * (warp - 4) + lane;
    const uint32_t lane_base = static_cast<uint32_t>(32 * (warp - 4)) << 16;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const float* src = tb + (part ? T.PhiL : T.PhiH);
      float v[KP];
#pragma unroll
      for (int j = 0; j < KP / 4; ++j) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(src + tc_canon(q, 4 * j, KP)));
        v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
      }
      tc::st_cols<KP>(tmem + lane_base + (part ? C::COL_PL : C::COL_PH), v);
    }
  }
  if (warp < 8) tc::wait_st();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  uint32_t phase = 0;
  bool failed = false;

  const int64_t ntiles = (a.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));
    __syncthreads();
    for (int w = tid; w < TE * QS / 4; w += blockDim.x) {
      const int e = w / (QS / 4), c = w - e * (QS / 4);
      if (e < ne) tc::cp_async16(sQ + e * QSP + 4 * c, a.q_in + (e0 + e) * QS + 4 * c);
      else *reinterpret_cast<float4*>(sQ + e * QSP + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int w = tid; w < TE * DS / 4; w += blockDim.x) {
      const int e = w / (DS / 4), c = w - e * (DS / 4);
      if (e < ne) tc::cp_async16(sD + e * DS + 4 * c, a.d + (e0 + e) * DS + 4 * c);
      else *reinterpret_cast<float4*>(sD + e * DS + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int w = tid; w < ne * 10; w += blockDim.x) {
      const int e = w / 10, k = w - 10 * e;
      if (k < 8) tc::cp_async16(sGM + e * 40 + 4 * k, reinterpret_cast<const float*>(a.geom + e0 + e) + 4 * k);
      else tc::cp_async16(sGM + e * 40 + 32 + 4 * (k - 8), reinterpret_cast<const float*>(a.mat + e0 + e) + 4 * (k - 8));
    }
    tc::cp_async_wait_all();
    __syncthreads();

#pragma unroll 1
    for (int iter = 0; iter < a.picard_iters && !failed; ++iter) {
      for (int w = tid; w < TE * DS; w += blockDim.x) sDn[w] = 0.f;
#pragma unroll 1
      for (int z = 0; z < NT; ++z) {
        // modal values of q(t_z) as the node-value MMA's B operand (row (element, field),
        // column mode); alpha to first order.  Lane (l mod 4, row mod 8): one core matrix per warp
        for (int w = tid; w < NU * KP; w += blockDim.x) {
          const int l4 = w & 3, n7 = (w >> 2) & 7, r = w >> 5;
          const int lq = r % (KP / 4), ng = r / (KP / 4);
          const int l = 4 * lq + l4, n = 8 * ng + n7, e = n / 12, c = n - 12 * e;
          float x = 0.f;
          if (e < TE && c < 10 && l < L) {
            const float* de = sD + e * DS;
            x = sQ[e * QSP + l * 10 + c];
            if (c < 9) {
#pragma unroll
              for (int o = 1; o <= N; ++o)
                if (l < n_modes(N - o)) x = fmaf(sCz[z * (N + 1) + o], de[d_offset(N, o) + l * 9 + c], x);
            } else {
              x = fmaf(sCz[z * (N + 1) + 1], de[AOFF + l], x);
            }
          }
          const int idx = tc_canon(n, l, KP);
          const float h = tc::tf32_hi(x);
          sBuH[idx] = h;
          sBuL[idx] = tc::tf32_hi(x - h);
        }
        tc::fence_smem_to_async();
        tc::fence_before();
        __syncthreads();
        if (tid == C::ISSUER) {
          tc::fence_after();
          constexpr uint32_t idesc = tc::idesc_tf32(128, NU);
          const uint32_t bH = tc::smem_u32(sBuH), bL = tc::smem_u32(sBuL);
#pragma unroll
          for (int ks = 0; ks < KP / 8; ++ks) {
            const uint32_t off = ks * 256;   // 8 K-elements = 2 core matrices
            const uint32_t aH = tmem + C::COL_PH + 8 * ks, aL = tmem + C::COL_PL + 8 * ks;
            tc::mma_tf32_ta(tmem + C::COL_U, aH, tc::desc_kmajor(bH + off, KP), idesc, ks > 0 ? 1u : 0u);
            tc::mma_tf32_ta(tmem + C::COL_U, aH, tc::desc_kmajor(bL + off, KP), idesc, 1u);
            tc::mma_tf32_ta(tmem + C::COL_U, aL, tc::desc_kmajor(bH + off, KP), idesc, 1u);
          }
          tc::commit(&mbar);
        }
        {
          const bool ok = tc::wait_parity(&mbar, phase, wait_limit);
          phase ^= 1u;
          if (__syncthreads_or(!ok)) {
            failed = true;
            break;
          }
        }
        tc::fence_after();
        // reference fluxes Theta^{-1}_{e'd} F^d and the damage rate at every node: warp group e
        // (warps 4e..4e+3) takes element e, thread q its volume node; the terms become the
        // projection's B operand less their value at node 0 (which returns through the row
        // sums of w_q phi_l(x_q))
        if (warp < 4 * TE) {
          const int e = warp >> 2, q = 32 * (warp & 3) + lane;
          const uint32_t lane_base = static_cast<uint32_t>(32 * (warp & 3)) << 16;
          float v[16];
          tc::ld_cols<16>(tmem + lane_base + C::COL_U + e * 12, v);
          tc::wait_ld();
          float out[28];
#pragma unroll
          for (int p = 0; p < 28; ++p) out[p] = 0.f;
          if (q < NQ && e < ne) {
            const float* gm = sGM + e * 40;
            const MatF m = *reinterpret_cast<const MatF*>(gm + 32);
            float sig[6], rr;
            law_point<LAW>(a.law, v, v[9], m, sig, &rr);
            const float S[3][3] = {{sig[0], sig[3], sig[5]}, {sig[3], sig[1], sig[4]}, {sig[5], sig[4], sig[2]}};
            const float vv[3] = {v[6], v[7], v[8]};
#pragma unroll
            for (int ep = 0; ep < 3; ++ep) {
              const float th[3] = {gm[ep * 3 + 0], gm[ep * 3 + 1], gm[ep * 3 + 2]};   // Theta^{-1}[e'][d]
              float* fe = out + ep * 9;
              fe[0] = -vv[0] * th[0];
              fe[1] = -vv[1] * th[1];
              fe[2] = -vv[2] * th[2];
              fe[3] = -0.5f * (vv[0] * th[1] + vv[1] * th[0]);
              fe[4] = -0.5f * (vv[1] * th[2] + vv[2] * th[1]);
              fe[5] = -0.5f * (vv[2] * th[0] + vv[0] * th[2]);
#pragma unroll
              for (int i = 0; i < 3; ++i) fe[6 + i] = -m.rho_inv * (S[i][0] * th[0] + S[i][1] * th[1] + S[i][2] * th[2]);
            }
            out[27] = rr;
          }
          if (q == 0) {
#pragma unroll
            for (int p = 0; p < 28; ++p) sC[e * 28 + p] = out[p];
          }
          tc::named_barrier(1 + e, 128);
          if (q < KQ) {
#pragma unroll
            for (int p = 0; p < 28; ++p) {
              const float x = q < NQ ? out[p] - sC[e * 28 + p] : 0.f;
              const int idx = C::prj_canon(e * 28 + p, q);
              const float h = tc::tf32_hi(x);
              sBfH[idx] = h;
              sBfL[idx] = tc::tf32_hi(x - h);
            }
          }
        }
        tc::fence_smem_to_async();
        tc::fence_before();
        __syncthreads();
        if (tid == C::ISSUER) {
          tc::fence_after();
          constexpr uint32_t idesc = tc::idesc_tf32(128, NPF);
          const uint32_t bH = tc::smem_u32(sBfH), bL = tc::smem_u32(sBfL);
          constexpr uint32_t lbo = 4u * C::PLBO, sbo = 4u * C::PGS;
#pragma unroll
          for (int ks = 0; ks < KQ / 8; ++ks) {
            const uint32_t off = ks * 2 * lbo;   // 8 K-elements = 2 core matrices
            const uint32_t aH = tmem + C::COL_AH + 8 * ks, aL = tmem + C::COL_AL + 8 * ks;
            tc::mma_tf32_ta(tmem + C::COL_F, aH, tc::desc_kmajor_strided(bH + off, lbo, sbo), idesc, ks > 0 ? 1u : 0u);
            tc::mma_tf32_ta(tmem + C::COL_F, aH, tc::desc_kmajor_strided(bL + off, lbo, sbo), idesc, 1u);
            tc::mma_tf32_ta(tmem + C::COL_F, aL, tc::desc_kmajor_strided(bH + off, lbo, sbo), idesc, 1u);
          }
          tc::commit(&mbar);
        }
        {
          const bool ok = tc::wait_parity(&mbar, phase, wait_limit);
          phase ^= 1u;
          if (__syncthreads_or(!ok)) {
            failed = true;
            break;
          }
        }
        tc::fence_after();
        // read-out: warps 0-3, lane = mode l; the node-0 values come back through the row sums
        if (warp < 4) {
          const int l = 32 * warp + lane;
          const uint32_t lane_base = static_cast<uint32_t>(32 * warp) << 16;
          const float sl = l < L ? __ldg(tb + T.PrjS + l) : 0.f;
#pragma unroll
          for (int c0 = 0; c0 < CF; c0 += 32) {
            float v[32];
            if (CF - c0 >= 32) tc::ld_x32(tmem + lane_base + C::COL_F + c0, v);
            else tc::ld_x16(tmem + lane_base + C::COL_F + c0, v);
            tc::wait_ld();
            if (l < L) {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (c0 + j < CF) sFh[l * CF + c0 + j] = fmaf(sC[c0 + j], sl, v[j]);
            }
          }
        }
        tc::fence_before();
        __syncthreads();
        // R(t_z) = -sum_e' Kt^{e'} Fh_{e'} + Shat, folded into the Taylor fit of every order;
        // items (mode, element, group of 3 fields)
        for (int w = tid; w < L * TE * 3; w += blockDim.x) {
          const int pg = w % 3, ke = w / 3;
          const int k = ke / TE, e = ke - k * TE;
          float* dn = sDn + e * DS;
          if (k < L1) {
            float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll 5
            for (int l = 0; l < L; ++l) {
              const float* fh = sFh + l * CF + e * 28 + 3 * pg;
#pragma unroll
              for (int ep = 0; ep < 3; ++ep) {
                const float kt = sKtA[(ep * L + l) * LP + k];
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[j] = fmaf(kt, fh[ep * 9 + j], acc[j]);
              }
            }
#pragma unroll
            for (int o = 1; o <= N; ++o) {
              if (k < n_modes(N - o)) {
#pragma unroll
                for (int j = 0; j < 3; ++j) dn[d_offset(N, o) + k * 9 + 3 * pg + j] -= sFit[(o - 1) * NT + z] * acc[j];
              }
            }
          }
          if (pg == 0) dn[AOFF + k] += sFit[z] * sFh[k * CF + e * 28 + 27];
        }
        __syncthreads();
      }
      if (failed) break;
      for (int w = tid; w < TE * DS; w += blockDim.x) sD[w] = sDn[w];
      __syncthreads();
    }
    if (failed) break;
    bool bad = false;
    for (int w = tid; w < ne * DS; w += blockDim.x) {
      bad |= !isfinite(sD[w]);
      a.d[e0 * DS + w] = sD[w];
    }
    if (bad) atomicOr(a.status, kStatusNonFinite);
  }
  if (failed) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    tc::wait_parity(&mbar, phase ^ 1u, kWaitLimit);   // let the MMAs in flight finish before freeing TMEM
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, C::TMEM_COLS);
}

// ===========================================================================
// Faces: Rusanov flux at the space-time nodes of each interior face, once per
// face; boundary faces (side 1 absent, tag in the fourth entry) take the
// absorbing or free-surface flux.  Persistent CTAs of 256 threads, two per SM.  Per tile of
// TF faces: both sides' state and predictor output staged in shared memory by
// one batch of asynchronous copies, with the per-face normal, speeds and
// materials; the traces as register-tiled products with the face basis table
// (G face nodes x 4 or 3 columns per thread, loops fully unrolled, warps 0-3
// on order 0 and warps 4-7 on orders >= 1, whose mode counts add up to about
// the same work); the flux at the face nodes with two threads per node, one per
// side.
// ===========================================================================
template <int N>
struct FluxCfg : Dim<N> {
  using D = Dim<N>;
  static constexpr int THREADS = 256;
  static constexpr int KT = THREADS / 2;                    // threads per trace kind
  static constexpr int G = N == 4 ? 5 : 4;                  // face nodes per trace tile
  static constexpr int NG = (D::NF + G - 1) / G;            // node groups
  static constexpr int NGG = NG * G;                        // padded face nodes
  static constexpr int GP = G == 5 ? 8 : 4;                 // stride of a node group in the table
  static constexpr int TF = KT / (6 * NG);                  // faces per tile: 2 TF NG 3 <= KT units per kind
  // lanes per face side in the trace phase: the side's NG * 3 units rounded up to a power
  // of two when the tile still fits, so that a warp's lanes cover whole sides (one local
  // face's table per half-warp at N = 4: 8% faster there)
  static constexpr int SPAN0 = NG * 3;
  static constexpr int SPANP = SPAN0 <= 4 ? 4 : (SPAN0 <= 8 ? 8 : (SPAN0 <= 16 ? 16 : 32));
  static constexpr int SPAN = 2 * TF * SPANP <= KT ? SPANP : SPAN0;
  static constexpr int UPK = 2 * TF * SPAN;                 // trace lanes per kind
  static constexpr int RAW_USED = D::QS + D::DS;            // staged floats per side: state, predictor output
  static constexpr int RAW = RAW_USED % 32 == 0 ? RAW_USED + 4 : RAW_USED;   // side stride off the bank period
  // node group g of a table row starts at g GP + 4 (g / (32 / GP)): groups that would
  // fall on the same banks are shifted by 16 bytes
  static constexpr int goff(int g) { return g * GP + 4 * (g / (32 / GP)); }
  static constexpr int VROW = round4(goff(NG - 1) + GP);
  // per face: n, |S|/|J|, cp-, cp+, tag, local faces, materials, side 0's mode-0 row
  static constexpr int META = 40;
  static constexpr int oV = 0;                              // [4][L][VROW] phi_l at the face nodes
  static constexpr int oRaw = round4(oV + 4 * D::L * VROW);  // [TF][2][RAW]
  static constexpr int oMeta = oRaw + TF * 2 * RAW;         // [2][TF][META], this tile's and the next one's
  static constexpr int oFR = oMeta + 2 * TF * META;         // [2][TF] int4 face records of the next two tiles
  static constexpr int oTr = round4(oFR + 2 * TF * 4);      // [TF][2][N+1][NGG][12] traces per order
  static constexpr int SMEM = oTr + TF * 2 * (N + 1) * NGG * 12;
  static_assert(TF >= 1 && UPK <= KT, "trace units per kind");
  static_assert(THREADS > 256 || SMEM * 4 * 2 <= 227 * 1024, "two face CTAs per SM");
};

template <int N>
__device__ __forceinline__ void load_group(const float* v, float* out) {
  using C = FluxCfg<N>;
  const float4 a = *reinterpret_cast<const float4*>(v);
  out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
  if constexpr (C::G == 5) out[4] = v[4];
}

// BND: the mesh has boundary faces (false compiles their flux out).
template <int N, int LAW, bool BND>
__global__ void __launch_bounds__(FluxCfg<N>::THREADS, 512 / FluxCfg<N>::THREADS) k_face_flux(StepArgs a) {
  using C = FluxCfg<N>;
  constexpr int L = C::L, NF = C::NF, NFP = C::NFP, NT = C::NT, QS = C::QS, DS = C::DS, AOFF = C::AOFF;
  constexpr int FFS = C::FFS, TF = C::TF, G = C::G, NG = C::NG, NGG = C::NGG, GP = C::GP, RAW = C::RAW;
  constexpr int META = C::META, UPK = C::UPK;
  constexpr TableLayout T = table_layout(N);
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* sV = sm + C::oV;
  float* sRaw = sm + C::oRaw;
  float* sMeta = sm + C::oMeta;
  float* sTr = sm + C::oTr;
  const float* tb = a.tables;
  const float dt = a.dt;
  const int tid = threadIdx.x;
  float tzs[NT], gzs[NT];                       // the time nodes and weights, scaled by dt
#pragma unroll
  for (int z = 0; z < NT; ++z) {
    tzs[z] = __ldg(tb + T.tz + z) * dt;
    gzs[z] = __ldg(tb + T.gz + z) * dt;
  }
  // face basis table regrouped by node groups (zero beyond the NF face nodes)
  for (int w = tid; w < 4 * L * NG * GP; w += C::THREADS) {
    const int n = w % GP, r = w / GP;
    const int g = r % NG, r2 = r / NG;
    const int l = r2 % L, lf = r2 / L;
    const int node = g * G + n;
    sV[(lf * L + l) * C::VROW + C::goff(g) + n] = (n < G && node < NF) ? __ldg(tb + T.VfT + (lf * L + l) * NFP + node) : 0.f;
  }

  // Copies of a tile's face data: per face the normal, both cells' P speeds and
  // materials (into the meta buffer mt0); per side the state and the predictor output
  // as stored (into sRaw).  Face records from fr (shared or global memory).
  const int64_t ntiles = (a.F + TF - 1) / TF;
  int4* sFR = reinterpret_cast<int4*>(sm + C::oFR);
  auto issue = [&](int64_t tl, const int4* fr, float* mt0, int t, int nt) {
    const int64_t f0 = tl * TF;
    const int nf = static_cast<int>(min(static_cast<int64_t>(TF), a.F - f0));
    constexpr int CH = C::RAW_USED / 4;          // 16-byte chunks per side
    for (int w = t; w < TF * (2 * CH + 8); w += nt) {
      const int fc = w / (2 * CH + 8), r = w - fc * (2 * CH + 8);
      if (fc >= nf) continue;
      const int4 fa = fr[fc];
      const bool bnd = fa.z < 0;
      if (r < 2 * CH) {
        const int side = r / CH, ch = r - side * CH;
        if (side && bnd) continue;
        const int64_t e = side ? fa.z : fa.x;
        float* dst = sRaw + (2 * fc + side) * RAW + 4 * ch;
        if (ch < QS / 4) tc::cp_async16(dst, a.q_in + e * QS + 4 * ch);
        else tc::cp_async16(dst, a.d + e * DS + 4 * (ch - QS / 4));
      } else {
        float* mt = mt0 + fc * META;
        const int k = r - 2 * CH;
        const int64_t ep = bnd ? fa.x : fa.z;
        if (k == 0) tc::cp_async16(mt, &a.geom[fa.x].face[fa.y][0]);
        else if (k == 1) tc::cp_async4(mt + 4, a.cp + fa.x);
        else if (k == 2) tc::cp_async4(mt + 5, a.cp + ep);
        else if (k == 3) {
          mt[6] = bnd ? static_cast<float>(fa.w) : 0.f;   // boundary tag
          mt[7] = static_cast<float>(fa.y);               // local face of side 0
          mt[24] = bnd ? 0.f : static_cast<float>(fa.w);  // local face of side 1
        } else {
          const int half = (k - 4) & 1, which = (k - 4) >> 1;
          tc::cp_async16(mt + 8 + 8 * which + 4 * half,
                         reinterpret_cast<const float*>(a.mat + (which ? ep : fa.x)) + 4 * half);
        }
      }
    }
  };
  // face records of tile tl into slot b
  auto issue_records = [&](int64_t tl, int b, int t, int nt) {
    const int64_t f0 = tl * TF;
    const int nf = static_cast<int>(min(static_cast<int64_t>(TF), a.F - f0));
    for (int w = t; w < nf; w += nt) tc::cp_async16(sFR + b * TF + w, a.faces + f0 + w);
  };

  if (static_cast<int64_t>(blockIdx.x) < ntiles)
    issue(blockIdx.x, a.faces + static_cast<int64_t>(blockIdx.x) * TF, sm + C::oMeta, tid, C::THREADS);
  if (static_cast<int64_t>(blockIdx.x) + gridDim.x < ntiles) issue_records(blockIdx.x + gridDim.x, 1, tid, C::THREADS);
  tc::cp_async_commit();
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t f0 = tile * TF;
    const int nf = static_cast<int>(min(static_cast<int64_t>(TF), a.F - f0));
    float* sMeta = sm + C::oMeta + (it & 1) * TF * META;
    __syncthreads();                           // the previous tile's flux phase is done
    tc::cp_async_wait<0>();                    // this tile's copies (and the next tile's face records)
    __syncthreads();
    // side 0's mode-0 row (the cell mean) for the boundary flux, kept with the face data:
    // the next tile's copies overwrite the state during the flux phase
    for (int w = tid; w < TF * 10; w += C::THREADS) {
      const int fc = w / 10, c = w - 10 * fc;
      sMeta[fc * META + 28 + c] = sRaw[(2 * fc) * RAW + c];
    }

    // traces: warps 0-3 order 0 (G nodes x 4 columns), warps 4-7 orders 1..N (G nodes x 3 fields)
    {
      const int kind = tid / C::KT, lu = tid - kind * C::KT;
      const int s2 = lu / C::SPAN, r = lu - s2 * C::SPAN;
      if (lu < UPK && r < NG * 3) {
        const int g = r / 3, c = r - 3 * g;
        const int fc = s2 >> 1, side = s2 & 1;
        const float* mt = sMeta + fc * META;
        if (fc < nf && !(side && BND && mt[6] != 0.f)) {
          const int lf = static_cast<int>(side ? mt[24] : mt[7]);
          const float* V = sV + lf * L * C::VROW + C::goff(g);
          const float* R = sRaw + s2 * RAW;
          float* out = sTr + (s2 * (N + 1)) * NGG * 12 + (g * G) * 12;
          if (kind == 0) {
            // columns 4c..4c+3 of (the ten fields, D^1 alpha, 0); the state is [L][10]
            const bool c2 = c == 2;
            const float* pB = c2 ? R + QS + AOFF : R + 4 * c + 2;
            const int sB = c2 ? 1 : 10, o3 = c2 ? 0 : 4 * c + 3;
            float acc[G][4];
#pragma unroll
            for (int n = 0; n < G; ++n)
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[n][j] = 0.f;
#pragma unroll
            for (int l = 0; l < L; ++l) {
              float v[G];
              load_group<N>(V + l * C::VROW, v);
              const float2 x01 = *reinterpret_cast<const float2*>(R + l * 10 + 4 * c);
              const float x2 = pB[l * sB], x3r = R[l * 10 + o3];
              const float x[4] = {x01.x, x01.y, x2, c2 ? 0.f : x3r};
#pragma unroll
              for (int n = 0; n < G; ++n)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[n][j] = fmaf(v[n], x[j], acc[n][j]);
            }
#pragma unroll
            for (int n = 0; n < G; ++n)
              *reinterpret_cast<float4*>(out + n * 12 + 4 * c) = make_float4(acc[n][0], acc[n][1], acc[n][2], acc[n][3]);
          } else {
            const float* Dh = R + QS + 3 * c;
#pragma unroll
            for (int o = 1; o <= N; ++o) {
              float acc[G][3];
#pragma unroll
              for (int n = 0; n < G; ++n)
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[n][j] = 0.f;
#pragma unroll
              for (int l = 0; l < n_modes(N - o); ++l) {
                float v[G];
                load_group<N>(V + l * C::VROW, v);
                const float* xr = Dh + d_offset(N, o) + l * 9;
                const float x[3] = {xr[0], xr[1], xr[2]};
#pragma unroll
                for (int n = 0; n < G; ++n)
#pragma unroll
                  for (int j = 0; j < 3; ++j) acc[n][j] = fmaf(v[n], x[j], acc[n][j]);
              }
              float* oo = out + o * NGG * 12 + 3 * c;
#pragma unroll
              for (int n = 0; n < G; ++n)
#pragma unroll
                for (int j = 0; j < 3; ++j) oo[n * 12 + j] = acc[n][j];
            }
          }
        }
      }
    }
    __syncthreads();
    // the next tile's copies (its face records landed with this tile's data), then the
    // records of the tile after it, while the flux runs
    if (tile + gridDim.x < ntiles)
      issue(tile + gridDim.x, sFR + ((it + 1) & 1) * TF, sm + C::oMeta + ((it + 1) & 1) * TF * META, tid, C::THREADS);
    if (tile + 2 * static_cast<int64_t>(gridDim.x) < ntiles)
      issue_records(tile + 2 * static_cast<int64_t>(gridDim.x), it & 1, tid, C::THREADS);
    tc::cp_async_commit();

    // flux at the face nodes, time-integrated.  The strain rows of the normal flux, the
    // Rusanov term and the whole boundary flux are linear in the state: their time integral
    // is their value at the time-integrated trace (the time rule integrates the degree-N
    // Taylor polynomial exactly).  Only the stress of the velocity rows is taken at the time
    // nodes.  Every part splits by side: of the two threads of a (face, node) pair, each
    // takes one side over all time nodes, and a shuffle adds the two.
    for (int w0 = 0; w0 < 2 * TF * NF; w0 += C::THREADS) {
      const int w = w0 + tid;
      const int pair = w >> 1, side = w & 1;
      const int fc = pair / NF, i = pair - fc * NF;
      float Fb[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) Fb[p] = 0.f;
      const float* mt = sMeta + fc * META;
      const int bc = (BND && fc < nf) ? static_cast<int>(mt[6]) : 0;
      if (fc < nf && (bc == 0 || side == 0)) {
        const float n[3] = {mt[0], mt[1], mt[2]};
        MatF m;
        {
          const float* m0 = mt + 8 + 8 * side;
          m.rho = m0[0]; m.lam0 = m0[1]; m.mu0 = m0[2]; m.gamma_r = m0[3];
          m.xi0 = m0[4]; m.cd = m0[5]; m.rho_inv = m0[6]; m.pad = 0.f;
        }
        const float* Tr = sTr + (2 * fc + side) * (N + 1) * NGG * 12 + i * 12;
        // the strain's Taylor coefficients, alpha and its rate, and the time-integrated
        // trace ub = sum_o D^o dt^(o+1) / (o+1)!
        float eo[N + 1][6], ub[9];
        float al, dal;
        {
          const float4 a0 = *reinterpret_cast<const float4*>(Tr);
          const float4 a1 = *reinterpret_cast<const float4*>(Tr + 4);
          const float4 a2 = *reinterpret_cast<const float4*>(Tr + 8);
          eo[0][0] = a0.x; eo[0][1] = a0.y; eo[0][2] = a0.z; eo[0][3] = a0.w; eo[0][4] = a1.x; eo[0][5] = a1.y;
          al = a2.y;
          dal = a2.z;
          const float u0[9] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x};
#pragma unroll
          for (int p = 0; p < 9; ++p) ub[p] = dt * u0[p];
        }
        float cw = dt;
#pragma unroll
        for (int o = 1; o <= N; ++o) {
          cw *= dt * (1.f / static_cast<float>(o + 1));   // constant after unrolling: no division
          const float* to = Tr + o * NGG * 12;
          const float4 b0 = *reinterpret_cast<const float4*>(to);
          const float4 b1 = *reinterpret_cast<const float4*>(to + 4);
          const float b2 = to[8];
          eo[o][0] = b0.x; eo[o][1] = b0.y; eo[o][2] = b0.z; eo[o][3] = b0.w; eo[o][4] = b1.x; eo[o][5] = b1.y;
          const float uo[9] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w, b2};
#pragma unroll
          for (int p = 0; p < 9; ++p) ub[p] = fmaf(cw, uo[p], ub[p]);
        }
        if (BND && bc != 0) {
          float lam, mu;
          effective_lame<LAW>(a.law, mt + 28, m, &lam, &mu);   // side 0's cell-mean modes
          const float cpb = sqrtf(fmaxf(lam + 2.f * mu, 0.f) * m.rho_inv);
          const float csb = sqrtf(fmaxf(mu, 0.f) * m.rho_inv);
          const float k_p = lam + 2.f * mu > 0.f ? cpb / (lam + 2.f * mu) : 0.f;
          boundary_flux(bc, ub, n, lam, mu, m.rho_inv, cpb, csb, k_p, Fb);
        } else {
          // this side's half of the strain rows and of the Rusanov term (+ for side 0)
          const float hc = (side ? -0.5f : 0.5f) * fmaxf(mt[4], mt[5]);
          Fb[0] = fmaf(hc, ub[0], -0.5f * ub[6] * n[0]);
          Fb[1] = fmaf(hc, ub[1], -0.5f * ub[7] * n[1]);
          Fb[2] = fmaf(hc, ub[2], -0.5f * ub[8] * n[2]);
          Fb[3] = fmaf(hc, ub[3], -0.25f * (ub[6] * n[1] + ub[7] * n[0]));
          Fb[4] = fmaf(hc, ub[4], -0.25f * (ub[7] * n[2] + ub[8] * n[1]));
          Fb[5] = fmaf(hc, ub[5], -0.25f * (ub[8] * n[0] + ub[6] * n[2]));
          Fb[6] = hc * ub[6];
          Fb[7] = hc * ub[7];
          Fb[8] = hc * ub[8];
          // this side's half of the velocity rows, -sigma n / rho, at the time nodes
          float sn[3] = {0.f, 0.f, 0.f};
#pragma unroll
          for (int z = 0; z < NT; ++z) {
            const float tau = tzs[z], gam = gzs[z];
            float e[6];
#pragma unroll
            for (int p = 0; p < 6; ++p) e[p] = eo[0][p];
            float c = 1.f;
#pragma unroll
            for (int o = 1; o <= N; ++o) {
              c *= tau * (1.f / static_cast<float>(o));
#pragma unroll
              for (int p = 0; p < 6; ++p) e[p] = fmaf(c, eo[o][p], e[p]);
            }
            float sig[6], r;
            law_point<LAW>(a.law, e, fmaf(tau, dal, al), m, sig, &r);
            sn[0] = fmaf(gam, sig[0] * n[0] + sig[3] * n[1] + sig[5] * n[2], sn[0]);
            sn[1] = fmaf(gam, sig[3] * n[0] + sig[1] * n[1] + sig[4] * n[2], sn[1]);
            sn[2] = fmaf(gam, sig[5] * n[0] + sig[4] * n[1] + sig[2] * n[2], sn[2]);
          }
          const float k = -0.5f * m.rho_inv;
          Fb[6] = fmaf(k, sn[0], Fb[6]);
          Fb[7] = fmaf(k, sn[1], Fb[7]);
          Fb[8] = fmaf(k, sn[2], Fb[8]);
        }
      }
#pragma unroll
      for (int p = 0; p < 9; ++p) Fb[p] += __shfl_down_sync(0xffffffffu, Fb[p], 1);
      if (fc < nf && side == 0) {
        float* out = a.ff + (f0 + fc) * FFS + i * 9;
#pragma unroll
        for (int p = 0; p < 9; ++p) out[p] = Fb[p];
      }
    }
  }
  tc::cp_async_wait<0>();                      // no copy may still be in flight at exit
}

// ===========================================================================
// Corrector: volume terms, face terms from the face fluxes, update
// ===========================================================================
// The velocity rows of the volume term, sum_q w_q d phi_k/d xi_e' (x_q) T_e'm(x_q),
// are taken as sum_l (int phi_l d phi_k/d xi_e') That_e'm,l with That the
// projection of T by the volume rule: d phi_k/d xi_e' has degree N-1, so the two
// agree up to rounding, and the same derivative table serves the strain rows.
template <int N, bool TSM>
struct CorrCfg : Dim<N> {
  using D = Dim<N>;
  static constexpr int TE = N >= 4 ? 4 : (N == 3 ? 8 : 16);
  static constexpr int THREADS = 256;
  static constexpr int NV = 3 * TE;                        // (element, component) columns
  static constexpr int NB = 10 * TE;                       // nodal columns (element, 9 stress terms + rate)
  static constexpr int NM = 2 * NV;                        // modal columns: time-integrated v | That_e'
  static constexpr int NFC = 9 * TE;                       // face columns (element, field)
  static constexpr int KS_PRJ = N >= 4 ? 2 : 1, KS_MOD = 1, KS_FACE = N >= 4 ? 2 : 1;
  // tables (only when TSM)
  static constexpr int oVvT = 0;
  static constexpr int oVw = TSM ? round4(oVvT + D::L * D::NQP) : 0;   // [NQ][LP]
  static constexpr int oKtB = TSM ? round4(oVw + D::NQ * D::LP) : 0;   // [3][L][LP]
  static constexpr int oVfw = TSM ? round4(oKtB + 3 * D::L * D::LP) : 0;   // [4 NF][LP]
  // element tile
  static constexpr int oQ = TSM ? round4(oVfw + 4 * D::NF * D::LP) : 0;   // [TE][QS]
  static constexpr int oC0 = oQ + TE * D::QS;              // [L][8 TE]  eps(6), alpha0, alpha1
  static constexpr int oCh = oC0 + D::L * 8 * TE;          // [SH][8 TE] higher-order strain rows
  static constexpr int BN = D::NQ * nb_stride(TE), BF = 4 * D::NF * NFC;
  static constexpr int oB = oCh + round4(D::SH) * 8 * TE;  // [NQ][NB] nodal terms | [4 NF][NFC] face fluxes
  static constexpr int oM = oB + round4(BN > BF ? BN : BF);     // [3][L][NM] modal GEMM inputs
  static constexpr int oA = oM + 3 * D::L * NM;            // [TE][L][10] update accumulator
  static constexpr int oH = oA + TE * D::L * 10;           // [3][LP][NM] modal GEMM outputs
  static constexpr int P1 = KS_PRJ * D::LP * NB, P2 = KS_FACE * D::LP * NFC;
  static constexpr int oPart = oH + 3 * D::LP * NM;
  static constexpr int SMEM = oPart + (P1 > P2 ? P1 : P2);
  static constexpr bool FITS = SMEM * 4 <= 227 * 1024;
  static_assert(FITS || TSM, "corrector shared memory");
};

// Second half of the corrector, shared by the SIMT and tensor-core variants:
// projection of the nodal terms (sB: [NQ][10 TE], columns (element, 9 stress
// terms T_e'm, integrated rate)) by the volume rule, modal derivative of the
// velocity and strain rows, face term from the face fluxes, update.  sM holds
// the time-integrated velocity in columns [0, 3 TE) of each [L][6 TE] block.
template <int N, int TE, int KS_PRJ, int KS_FACE>
__device__ __forceinline__ void corrector_tail(const StepArgs& a, int64_t e0, int ne, const float* sVw,
                                               const float* sKtB, const float* sVfw, const float* sQ, float* sM,
                                               float* sB, float* sA, float* sH, float* sPart,
                                               const float* sFraw = nullptr, const float* sGeo = nullptr) {
  using D = Dim<N>;
  constexpr int L = D::L, NQ = D::NQ, NF = D::NF, LP = D::LP, QS = D::QS, FFS = D::FFS;
  constexpr int NV = 3 * TE, NB = 10 * TE, NM = 2 * NV, NFC = 9 * TE;
    // projection by the volume rule: That_e'm (into the modal inputs) and the damage source
    block_gemm<KS_PRJ>(sVw, LP, sB, nb_stride(TE), LP, NB, NQ, sPart, [&](int l, int col, float v) {
      if (l < L) {
        const int e = col / 10, c = col - 10 * e;
        if (c < 9) sM[((c / 3) * L + l) * NM + NV + e * 3 + c % 3] = v;
        else sA[(e * L + l) * 10 + 9] += v;
      }
    });
    if (KS_PRJ == 1) __syncthreads();
    // modal derivative: H_e'[k][col] = sum_l int phi_l d phi_k/d xi_e' M_e'[l][col], e' = 0..2 in one pass
    {
      constexpr int MQ = LP / 4, NQQ = NM / 4, TILES = MQ * NQQ;
      for (int w = threadIdx.x; w < 3 * TILES; w += blockDim.x) {
        const int ep = w / TILES, r = w - ep * TILES;
        const int ni = r % NQQ, mi = r / NQQ;   // column quad fastest: contiguous stores
        const float* A = sKtB + ep * L * LP + 4 * mi;
        const float* B = sM + ep * L * NM + 4 * ni;
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 5
        for (int l = 0; l < L; ++l) {
          const float4 av = *reinterpret_cast<const float4*>(A + l * LP);
          const float4 bv = *reinterpret_cast<const float4*>(B + l * NM);
          const float x[4] = {av.x, av.y, av.z, av.w}, y[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(x[i], y[j], acc[i][j]);
        }
        float* h = sH + ep * LP * NM;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          *reinterpret_cast<float4*>(h + (4 * mi + i) * NM + 4 * ni) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      }
    }
    // face fluxes of the tile's elements, signed and scaled by |S_f| / |J| (sB is free again)
    for (int w = threadIdx.x; w < TE * 4 * NF * 9; w += blockDim.x) {
      const int e = w / (4 * NF * 9), r = w - e * 4 * NF * 9;
      const int f = r / (NF * 9), r2 = r - f * NF * 9;
      const int i = r2 / 9, p = r2 - 9 * i;
      float v = 0.f;
      if (e < ne) {
        if (sFraw) {
          v = sGeo[e * 32 + 17 + f] * sFraw[(e * 4 + f) * FFS + i * 9 + p];
        } else {
          const int64_t ge = e0 + e;
          const int ef = a.elem_face[ge * 4 + f];
          const float sc = a.geom[ge].face[f][3] * ((ef & 1) ? -1.f : 1.f);
          v = sc * __ldg(a.ff + static_cast<int64_t>(ef >> 1) * FFS + i * 9 + p);
        }
      }
      sB[(f * NF + i) * NFC + e * 9 + p] = v;
    }
    __syncthreads();
    // strain rows -(v_i d_j phi + v_j d_i phi)/2 and velocity rows from the modal derivatives
    for (int w = threadIdx.x; w < TE * L; w += blockDim.x) {
      const int k = w / TE, e = w - k * TE;     // element fastest: lanes spread over the banks of sH
      const float* ti = sGeo ? sGeo + e * 32 : a.geom[e0 + (e < ne ? e : 0)].tinv;
      float hd[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int mc = 0; mc < 3; ++mc)
          hd[d][mc] = ti[0 * 3 + d] * sH[(0 * LP + k) * NM + e * 3 + mc] + ti[1 * 3 + d] * sH[(1 * LP + k) * NM + e * 3 + mc] +
                      ti[2 * 3 + d] * sH[(2 * LP + k) * NM + e * 3 + mc];
      float* ao = sA + (e * L + k) * 10;
      ao[0] -= hd[0][0];
      ao[1] -= hd[1][1];
      ao[2] -= hd[2][2];
      ao[3] -= 0.5f * (hd[1][0] + hd[0][1]);
      ao[4] -= 0.5f * (hd[2][1] + hd[1][2]);
      ao[5] -= 0.5f * (hd[0][2] + hd[2][0]);
#pragma unroll
      for (int mc = 0; mc < 3; ++mc)
        ao[6 + mc] += sH[(0 * LP + k) * NM + NV + e * 3 + mc] + sH[(1 * LP + k) * NM + NV + e * 3 + mc] +
                      sH[(2 * LP + k) * NM + NV + e * 3 + mc];
    }
    __syncthreads();
    block_gemm<KS_FACE>(sVfw, LP, sB, NFC, LP, NFC, 4 * NF, sPart, [&](int k, int col, float v) {
      if (k < L) {
        const int e = col / 9, p = col - 9 * e;
        sA[(e * L + k) * 10 + p] -= v;
      }
    });
    if (KS_FACE == 1) __syncthreads();
    // update
    bool bad = false;
    for (int w = threadIdx.x; w < ne * L * 10; w += blockDim.x) {
      const int e = w / (L * 10), r = w - e * (L * 10);
      const float v = sQ[e * QS + r] + sA[e * L * 10 + r];
      bad |= !isfinite(v);
      a.q_out[(e0 + e) * QS + r] = v;
    }
    if (bad) atomicOr(a.status, kStatusNonFinite);
}

// Phases of the tensor-core corrector that run on the SIMT cores while an MMA is in
// flight.  The modal derivative takes one half of the modal inputs at a time:
// H_e'[k][c0 + j] = sum_l int phi_l d phi_k / d xi_e' M_e'[l][c0 + j], e' = 0..2,
// j < 3 TE (c0 = 0: time-integrated velocity, c0 = 3 TE: the projected terms That).
template <int N, int TE>
__device__ __forceinline__ void modal_derivative_half(const float* sKtB, const float* sM, float* sH, int c0, int t,
                                                      int nt) {
  using D = Dim<N>;
  constexpr int L = D::L, LP = D::LP, NV = 3 * TE, NM = 2 * NV;
  constexpr int MQ = LP / 4, NP = NV / 2, TILES = MQ * NP;   // 4 rows x 2 columns per thread
  for (int w = t; w < 3 * TILES; w += nt) {
    const int ep = w / TILES, r = w - ep * TILES;
    const int mi = r / NP, ni = r - mi * NP;
    const float* A = sKtB + ep * L * LP + 4 * mi;
    const float* B = sM + ep * L * NM + c0 + 2 * ni;
    float acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = 0.f;
#pragma unroll 5
    for (int l = 0; l < L; ++l) {
      const float4 av = *reinterpret_cast<const float4*>(A + l * LP);
      const float2 bv = *reinterpret_cast<const float2*>(B + l * NM);
      const float x[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] = fmaf(x[i], bv.x, acc[i][0]);
        acc[i][1] = fmaf(x[i], bv.y, acc[i][1]);
      }
    }
    float* h = sH + ep * LP * NM + c0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      *reinterpret_cast<float2*>(h + (4 * mi + i) * NM + 2 * ni) = make_float2(acc[i][0], acc[i][1]);
  }
}

// Strain rows -(v_i d_j phi + v_j d_i phi)/2 from the velocity half of H (element fastest:
// the lanes of a warp spread over the banks of sH).
template <int N, int TE>
__device__ __forceinline__ void strain_rows(const float* sH, const float* sGeo, float* sA, int t, int nt) {
  using D = Dim<N>;
  constexpr int L = D::L, LP = D::LP, NM = 6 * TE;
  for (int w = t; w < TE * L; w += nt) {
    const int k = w / TE, e = w - k * TE;
    const float* ti = sGeo + e * 32;
    float hd[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int mc = 0; mc < 3; ++mc)
        hd[d][mc] = ti[0 * 3 + d] * sH[(0 * LP + k) * NM + e * 3 + mc] + ti[1 * 3 + d] * sH[(1 * LP + k) * NM + e * 3 + mc] +
                    ti[2 * 3 + d] * sH[(2 * LP + k) * NM + e * 3 + mc];
    float* ao = sA + (e * L + k) * 10;
    ao[0] -= hd[0][0];
    ao[1] -= hd[1][1];
    ao[2] -= hd[2][2];
    ao[3] -= 0.5f * (hd[1][0] + hd[0][1]);
    ao[4] -= 0.5f * (hd[2][1] + hd[1][2]);
    ao[5] -= 0.5f * (hd[0][2] + hd[2][0]);
  }
}

// Velocity rows: the sum over e' of the That half of H.
template <int N, int TE>
__device__ __forceinline__ void velocity_rows(const float* sH, float* sA) {
  using D = Dim<N>;
  constexpr int L = D::L, LP = D::LP, NV = 3 * TE, NM = 2 * NV;
  for (int w = threadIdx.x; w < TE * L; w += blockDim.x) {
    const int k = w / TE, e = w - k * TE;
    float* ao = sA + (e * L + k) * 10;
#pragma unroll
    for (int mc = 0; mc < 3; ++mc)
      ao[6 + mc] += sH[(0 * LP + k) * NM + NV + e * 3 + mc] + sH[(1 * LP + k) * NM + NV + e * 3 + mc] +
                    sH[(2 * LP + k) * NM + NV + e * 3 + mc];
  }
}

template <int N, bool TSM, int LAW>
__global__ void __launch_bounds__(256) k_corrector(StepArgs a) {
  using C = CorrCfg<N, TSM>;
  constexpr int L = C::L, NQ = C::NQ, NQP = C::NQP, NF = C::NF, NT = C::NT, LP = C::LP;
  constexpr int QS = C::QS, DS = C::DS, AOFF = C::AOFF, TE = C::TE;
  constexpr int NM = C::NM;
  constexpr TableLayout T = table_layout(N);
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const float* sVvT = TSM ? sm + C::oVvT : a.tables + T.VvT;
  const float* sVw = TSM ? sm + C::oVw : a.tables + T.Vw;
  const float* sKtB = TSM ? sm + C::oKtB : a.tables + T.KtB;
  const float* sVfw = TSM ? sm + C::oVfw : a.tables + T.Vfw;
  float* sQ = sm + C::oQ;
  float* sC0 = sm + C::oC0;
  float* sCh = sm + C::oCh;
  float* sB = sm + C::oB;
  float* sM = sm + C::oM;
  float* sA = sm + C::oA;
  float* sH = sm + C::oH;
  float* sPart = sm + C::oPart;
  const float* tb = a.tables;
  const float dt = a.dt;
  if (TSM) {
    copy_to_smem(sm + C::oVvT, tb + T.VvT, L * NQP);
    copy_to_smem(sm + C::oVw, tb + T.Vw, NQ * LP);
    copy_to_smem(sm + C::oKtB, tb + T.KtB, 3 * L * LP);
    copy_to_smem(sm + C::oVfw, tb + T.Vfw, 4 * NF * LP);
  }
  float tz[NT], gz[NT];
#pragma unroll
  for (int z = 0; z < NT; ++z) {
    tz[z] = __ldg(tb + T.tz + z) * dt;
    gz[z] = __ldg(tb + T.gz + z) * dt;
  }

  const int64_t ntiles = (a.E + TE - 1) / TE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e0 = tile * TE;
    const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));
    __syncthreads();
    {
      const float4* src = reinterpret_cast<const float4*>(a.q_in + e0 * QS);
      float4* dst = reinterpret_cast<float4*>(sQ);
      for (int w = threadIdx.x; w < TE * QS / 4; w += blockDim.x)
        dst[w] = w < ne * QS / 4 ? __ldg(src + w) : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int w = threadIdx.x; w < TE * L * 10; w += blockDim.x) sA[w] = 0.f;
    }
    __syncthreads();
    // coefficient arrays of the volume evaluation and the time-integrated velocity
    for (int w = threadIdx.x; w < L * TE; w += blockDim.x) {
      const int l = w / TE, e = w - l * TE;
      const float* q = sQ + e * QS + l * 10;
      const bool live = e < ne;
      const float* de = a.d + (e0 + (live ? e : 0)) * DS;
      float* c0 = sC0 + l * 8 * TE + e * 8;
#pragma unroll
      for (int p = 0; p < 6; ++p) c0[p] = q[p];
      c0[6] = q[9];
      c0[7] = live ? __ldg(de + AOFF + l) : 0.f;
      float iv[3] = {dt * q[6], dt * q[7], dt * q[8]};
      float c = dt;
#pragma unroll
      for (int o = 1; o <= N; ++o) {
        c *= dt * (1.f / static_cast<float>(o + 1));
        if (l < n_modes(N - o)) {
          const float* dd = de + d_offset(N, o) + l * 9;
          float* ch = sCh + (row_hi(N, o) + l) * 8 * TE + e * 8;
#pragma unroll
          for (int p = 0; p < 6; ++p) ch[p] = live ? __ldg(dd + p) : 0.f;
          ch[6] = ch[7] = 0.f;
#pragma unroll
          for (int m = 0; m < 3; ++m) iv[m] = fmaf(c, live ? __ldg(dd + 6 + m) : 0.f, iv[m]);
        }
      }
#pragma unroll
      for (int ep = 0; ep < 3; ++ep)
#pragma unroll
        for (int m = 0; m < 3; ++m) sM[(ep * L + l) * NM + e * 3 + m] = iv[m];
    }
    __syncthreads();

    // volume nodes: strains and damage in time, CDM stress and rate, time integral
    constexpr int NPAIR = NQP / 2;
    for (int w = threadIdx.x; w < TE * NPAIR; w += blockDim.x) {
      const int e = w / NPAIR, j = w - e * NPAIR;
      float a0[2][8];
      float ah[N][2][6];
#pragma unroll
      for (int n = 0; n < 2; ++n) {
#pragma unroll
        for (int p = 0; p < 8; ++p) a0[n][p] = 0.f;
#pragma unroll
        for (int o = 0; o < N; ++o)
#pragma unroll
          for (int p = 0; p < 6; ++p) ah[o][n][p] = 0.f;
      }
#pragma unroll 5
      for (int l = 0; l < L; ++l) {
        const float2 ph = *reinterpret_cast<const float2*>(sVvT + l * NQP + 2 * j);
        const float4 c0 = *reinterpret_cast<const float4*>(sC0 + l * 8 * TE + e * 8);
        const float4 c1 = *reinterpret_cast<const float4*>(sC0 + l * 8 * TE + e * 8 + 4);
        const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          a0[0][p] = fmaf(ph.x, cv[p], a0[0][p]);
          a0[1][p] = fmaf(ph.y, cv[p], a0[1][p]);
        }
      }
#pragma unroll
      for (int o = 1; o <= N; ++o) {
        const int rb = row_hi(N, o);
#pragma unroll 4
        for (int l = 0; l < n_modes(N - o); ++l) {
          const float2 ph = *reinterpret_cast<const float2*>(sVvT + l * NQP + 2 * j);
          const float4 c0 = *reinterpret_cast<const float4*>(sCh + (rb + l) * 8 * TE + e * 8);
          const float2 c1 = *reinterpret_cast<const float2*>(sCh + (rb + l) * 8 * TE + e * 8 + 4);
          const float cv[6] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y};
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            ah[o - 1][0][p] = fmaf(ph.x, cv[p], ah[o - 1][0][p]);
            ah[o - 1][1][p] = fmaf(ph.y, cv[p], ah[o - 1][1][p]);
          }
        }
      }
      const bool live = e < ne;
      const int64_t ge = e0 + (live ? e : 0);
      const MatF m = a.mat[ge];
      const float* ti = a.geom[ge].tinv;
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const int q = 2 * j + n;
        if (q >= NQ) continue;
        float sb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, rb = 0.f;
#pragma unroll
        for (int z = 0; z < NT; ++z) {
          float eps[6];
#pragma unroll
          for (int p = 0; p < 6; ++p) eps[p] = a0[n][p];
          float c = 1.f;
#pragma unroll
          for (int o = 1; o <= N; ++o) {
            c *= tz[z] * (1.f / static_cast<float>(o));
#pragma unroll
            for (int p = 0; p < 6; ++p) eps[p] = fmaf(c, ah[o - 1][n][p], eps[p]);
          }
          const float alpha = fmaf(tz[z], a0[n][7], a0[n][6]);
          float sig[6], r;
          law_point<LAW>(a.law, eps, alpha, m, sig, &r);
#pragma unroll
          for (int p = 0; p < 6; ++p) sb[p] = fmaf(gz[z], sig[p], sb[p]);
          rb = fmaf(gz[z], r, rb);
        }
        // T_e'm = -(1/rho) sum_d Theta^{-1}_{e'd} sigma_md (time integrated) and the integrated rate
        const float S[3][3] = {{sb[0], sb[3], sb[5]}, {sb[3], sb[1], sb[4]}, {sb[5], sb[4], sb[2]}};
        float* bq = sB + q * nb_stride(TE) + e * 10;
#pragma unroll
        for (int ep = 0; ep < 3; ++ep)
#pragma unroll
          for (int mc = 0; mc < 3; ++mc)
            bq[ep * 3 + mc] =
                live ? -m.rho_inv * (ti[ep * 3 + 0] * S[mc][0] + ti[ep * 3 + 1] * S[mc][1] + ti[ep * 3 + 2] * S[mc][2])
                     : 0.f;
        bq[9] = live ? rb : 0.f;
      }
    }
    __syncthreads();
    corrector_tail<N, TE, C::KS_PRJ, C::KS_FACE>(a, e0, ne, sVw, sKtB, sVfw, sQ, sM, sB, sA, sH, sPart);
  }
}

// ===========================================================================
// Corrector with the volume evaluation on the tensor cores (degrees 2..4)
// ===========================================================================
// The Taylor expansion at the N+1 time nodes, U(t_z) = sum_i t_z^i/i! D^i, is
// formed modally per element (columns (element, time node, eps_xx..eps_zx,
// alpha, 0)); one tcgen05 GEMM with the basis table as the 128 x KP operand
// gives every column at every volume node in TMEM, in 3xTF32 (TF32 high parts
// and FP32 remainders of both operands: FP32-level accuracy).  Thread q of
// warps w and w+4 owns TMEM lane (volume node) q and reads its columns.
template <int N>
struct CorrTcCfg : Dim<N> {
  using D = Dim<N>;
  static constexpr int TE = 4;
  static constexpr int THREADS = 512;                      // 16 warps (the item maps below assume it)
  static constexpr int GROUPS = THREADS / 128;             // warp groups reading TMEM (4 warps each)
  static constexpr int KP = tc_kp(N);
  static constexpr int KQ = tc_kq(N);                      // K of the projection (volume nodes, padded)
  static constexpr int NCOL = D::NT * 8;                   // columns per element
  static constexpr int NBC = TE * NCOL;                    // MMA N of the volume evaluation
  static constexpr int NV = 3 * TE, NB = 10 * TE, NM = 2 * NV, NFC = 9 * TE;
  static constexpr int NPC = (NB + 15) / 16 * 16;          // MMA N of the projection
  static constexpr int KS_FACE = N >= 4 ? 4 : 1, NJ_FACE = N >= 4 ? 3 : 2;   // face GEMM: k-split, columns per item
  // tensor memory: volume-node values (then the projection's D) | projection A (TF32
  // high part, remainder) | volume A phi_l(x_q) (TF32 high part, remainder)
  static constexpr int COL_DP = 0;
  static constexpr int COL_AH = (NBC + 31) / 32 * 32, COL_AL = COL_AH + KQ;
  static constexpr int COL_PH = COL_AL + KQ, COL_PL = COL_PH + KP;
  static constexpr int TMEM_NEED = COL_PL + KP;
  static constexpr int TMEM_COLS = TMEM_NEED <= 128 ? 128 : (TMEM_NEED <= 256 ? 256 : 512);
  static constexpr int oKtB = 0;
  static constexpr int oVfw = round4(oKtB + 3 * D::L * D::LP);
  // GEMM operand region (TF32 high parts and remainders): the volume operand [NBC x KP],
  // then the projection operand [NPC x KQ] (the nodal terms)
  // The projection operand's core matrices are 36 floats apart along K (4 floats of
  // padding), so that the 32 volume nodes written by one warp land in 32 banks.
  static constexpr int PLBO = 36, PGS = KQ / 4 * PLBO, BP = NPC / 8 * PGS;
  static constexpr int oBeH = round4(oVfw + 4 * D::NF * D::LP);
  static constexpr int BE_SIZE = (2 * NBC * KP > 2 * BP ? 2 * NBC * KP : 2 * BP);
  static constexpr int BE_END = oBeH + BE_SIZE;
  static constexpr int oBeL = oBeH + NBC * KP;
  static constexpr int oBpH = oBeH, oBpL = oBeH + BP;
  // outside the operand region, for the phases that overlap an MMA: modal outputs,
  // scaled face fluxes, the face GEMM's partial sums
  static constexpr int oH = BE_END;                        // [3][LP][NM]
  static constexpr int oF = round4(oH + 3 * D::LP * NM);   // [4 NF][NFC]
  static constexpr int oPart = round4(oF + 4 * D::NF * NFC);
  static constexpr int oM = oPart + KS_FACE * D::LP * NFC; // [3][L][NM] modal GEMM inputs
  static constexpr int oA = oM + 3 * D::L * NM;            // [TE][L][10] update accumulator
  // two tile buffers filled by asynchronous copies (the next tile's while this one computes):
  // state, predictor output, face fluxes, GeomF, MatF, face ids, and the face ids of
  // the CTA's tile after that one (whose face fluxes the next copy fetches)
  static constexpr int bQ = 0, bD = TE * D::QS, bF = bD + TE * D::DS, bG = bF + TE * 4 * D::FFS;
  static constexpr int bM = bG + TE * 32, bE = bM + TE * 8, bI = bE + TE * 4;
  static constexpr int BUF = bI + TE * 4;
  static_assert(D::QS % 4 == 0 && D::DS % 4 == 0 && D::FFS % 4 == 0 && sizeof(GeomF) == 128 && sizeof(MatF) == 32,
                "16-byte copies");
  static constexpr int oBuf = round4(oA + TE * D::L * 10);
  static constexpr int oGeo = oBuf + 2 * BUF;              // [TE][32]: Theta^{-1}, material, face scales
  static constexpr int oC = oGeo + TE * 32;                // [TE][10] nodal terms at node 0
  // the last warp issues the MMAs; the others (the workers) run the SIMT phases meanwhile
  static constexpr int WORKERS = THREADS - 32, ISSUER = THREADS - 32;
  static constexpr int SMEM = round4(oC + TE * 10);
  static_assert(D::NQ <= 128 && NBC % 16 == 0 && NBC <= 256 && NPC <= 256 && KQ % 32 == 0, "tensor-core shapes");
  static_assert(D::L <= 64 && NB <= 40 && NB % 8 == 0 && TE * 4 <= THREADS / 32, "projection read-out: warps 0, 1 of each group");
  static_assert(THREADS == 512 && 21 * TE <= 128, "work maps of the tile's first stage");
  static_assert(NPC <= NBC && KP <= 40, "projection D inside the volume D; volume A in one row of stores");
  __host__ __device__ static constexpr int prj_canon(int n, int q) {
    return (n >> 3) * PGS + (q >> 2) * PLBO + (n & 7) * 4 + (q & 3);
  }
  static_assert(TMEM_NEED <= 512, "tensor memory columns");
  static_assert(SMEM * 4 <= 227 * 1024, "tensor-core corrector shared memory");
};

template <int N, int LAW>
__global__ void __launch_bounds__(CorrTcCfg<N>::THREADS, 1) k_corrector_tc(StepArgs a) {
  using C = CorrTcCfg<N>;
  constexpr int L = C::L, NQ = C::NQ, NF = C::NF, NT = C::NT, LP = C::LP, QS = C::QS, DS = C::DS;
  constexpr int AOFF = C::AOFF, TE = C::TE, KP = C::KP, KQ = C::KQ, NCOL = C::NCOL, NBC = C::NBC, NM = C::NM;
  constexpr int NV = C::NV, NPC = C::NPC, NFC = C::NFC;
  constexpr TableLayout T = table_layout(N);
  constexpr int kWaitLimit = 1 << 24;
  // the limit of the waits on the MMAs; the drain after a failure keeps the default
  const int wait_limit = a.wait_limit_set ? a.wait_limit : kWaitLimit;
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const float* sKtB = sm + C::oKtB;
  const float* sVfw = sm + C::oVfw;
  float* sBeH = sm + C::oBeH;
  float* sBeL = sm + C::oBeL;
  float* sM = sm + C::oM;
  float* sBpH = sm + C::oBpH;
  float* sBpL = sm + C::oBpL;
  float* sF = sm + C::oF;
  float* sC = sm + C::oC;
  float* sA = sm + C::oA;
  float* sH = sm + C::oH;
  float* sPart = sm + C::oPart;
  float* sGeo = sm + C::oGeo;
  constexpr int FFS = C::FFS;
  const float* tb = a.tables;
  const float dt = a.dt;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  copy_to_smem(sm + C::oKtB, tb + T.KtB, 3 * L * LP);
  copy_to_smem(sm + C::oVfw, tb + T.Vfw, 4 * NF * LP);
  float tz[NT], gz[NT];
#pragma unroll
  for (int z = 0; z < NT; ++z) {
    tz[z] = __ldg(tb + T.tz + z) * dt;
    gz[z] = __ldg(tb + T.gz + z) * dt;
  }
  if (warp == 0) tc::alloc(&tmem_base, C::TMEM_COLS);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  // projection operand A = w_q phi_l(x_q) (TF32 part, remainder) into tensor memory
  // once: lane l, columns q.  Warp w of the first group writes lanes [32 w, 32 w + 32).
  if (warp < 4) {
    const uint32_t lane_base = static_cast<uint32_t>(32 * warp) << 16;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const float* src = tb + (part ? T.PrjL : T.PrjH) + (32 * warp + lane) * KQ;
#pragma unroll 1
      for (int c0 = 0; c0 < KQ; c0 += 32) {
        float v[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 x = __ldg(reinterpret_cast<const float4*>(src + c0) + j);
          v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
        }
        tc::st_x32(tmem + lane_base + (part ? C::COL_AL : C::COL_AH) + c0, v);
      }
    }
  } else if (warp < 8) {
    // volume operand A = phi_l(x_q) (TF32 part, remainder): lane q, columns l, read from
    // the canonical tables (four consecutive l of a node are contiguous)
    const int q = 32 * (warp - 4) + lane;
    const uint32_t lane_base = static_cast<uint32_t>(32 * (warp - 4)) << 16;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      const float* src = tb + (part ? T.PhiL : T.PhiH);
      float v[KP];
#pragma unroll
      for (int j = 0; j < KP / 4; ++j) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(src + tc_canon(q, 4 * j, KP)));
        v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
      }
      tc::st_cols<KP>(tmem + lane_base + (part ? C::COL_PL : C::COL_PH), v);
    }
  }
  if (warp < 8) tc::wait_st();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  uint32_t phase = 0;
  bool failed = false;

  // one batch of 16-byte asynchronous copies of a tile on threads t of [0, nt): state,
  // predictor output, face fluxes (at the face ids `ids` of the tile), GeomF, MatF, face
  // ids, and the face ids of this CTA's following tile
  const int64_t ntiles = (a.E + TE - 1) / TE;
  auto issue = [&](int64_t tl, float* buf, const int* ids, int t, int nt) {
    const int64_t e0 = tl * TE;
    const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));
    const int64_t n0 = (tl + gridDim.x) * TE;
    const int nn = n0 < a.E ? static_cast<int>(min(static_cast<int64_t>(TE), a.E - n0)) : 0;
    for (int w = t; w < ne * QS / 4; w += nt) tc::cp_async16(buf + C::bQ + 4 * w, a.q_in + e0 * QS + 4 * w);
    for (int w = t; w < ne * DS / 4; w += nt) tc::cp_async16(buf + C::bD + 4 * w, a.d + e0 * DS + 4 * w);
    for (int w = t; w < ne * FFS; w += nt) {     // ne * 4 faces * FFS/4 chunks
      const int e = w / FFS, r = w - e * FFS;
      const int f = r / (FFS / 4), c = r - f * (FFS / 4);
      const int64_t fid = ids[e * 4 + f] >> 1;
      tc::cp_async16(buf + C::bF + (e * 4 + f) * FFS + 4 * c, a.ff + fid * FFS + 4 * c);
    }
    for (int w = t; w < ne * 11 + nn; w += nt) {
      if (w >= ne * 11) {
        tc::cp_async16(buf + C::bI + 4 * (w - ne * 11), a.elem_face + (n0 + w - ne * 11) * 4);
        continue;
      }
      const int e = w / 11, k = w - 11 * e;
      if (k < 8) tc::cp_async16(buf + C::bG + e * 32 + 4 * k, reinterpret_cast<const float*>(a.geom + e0 + e) + 4 * k);
      else if (k < 10) tc::cp_async16(buf + C::bM + e * 8 + 4 * (k - 8), reinterpret_cast<const float*>(a.mat + e0 + e) + 4 * (k - 8));
      else tc::cp_async16(buf + C::bE + e * 4, a.elem_face + (e0 + e) * 4);
    }
  };

  if (static_cast<int64_t>(blockIdx.x) < ntiles)
    issue(blockIdx.x, sm + C::oBuf, a.elem_face + static_cast<int64_t>(blockIdx.x) * TE * 4, tid, blockDim.x);
  tc::cp_async_commit();
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t e0 = tile * TE;
    const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));
    float* buf = sm + C::oBuf + (it & 1) * C::BUF;
    float* sQ = buf + C::bQ;
    const float* sDraw = buf + C::bD;
    const float* sFraw = buf + C::bF;
    const float* sGraw = buf + C::bG;
    __syncthreads();                         // the previous tile is done with every buffer
    tc::cp_async_wait<0>();                  // this tile's copies have landed
    for (int w = ne * QS + tid; w < TE * QS; w += blockDim.x) sQ[w] = 0.f;
    for (int w = tid; w < TE * L * 10; w += blockDim.x) sA[w] = 0.f;
    __syncthreads();
    // per element: Theta^{-1} [0,9), material [9,17), signed |S_f|/|J| [17,21)
    for (int w = tid; w < TE * 21; w += blockDim.x) {
      const int e = w / 21, c = w - 21 * e;
      const float* g = sGraw + e * 32;
      float v = 0.f;
      if (e < ne) {
        if (c < 9) {
          v = g[c];
        } else if (c < 17) {
          v = buf[C::bM + e * 8 + c - 9];
        } else {
          const int f = c - 17;
          v = g[12 + 4 * f + 3] * ((__float_as_int(buf[C::bE + e * 4 + f]) & 1) ? -1.f : 1.f);
        }
      }
      sGeo[e * 32 + c] = v;
    }
    // time-integrated velocity (modal), the first 3 TE columns of each [L][NM] block of sM,
    // on threads from 128 on (the per-element data above runs on the first ones)
    for (int w = (tid + C::THREADS - 128) % C::THREADS; w < L * TE; w += blockDim.x) {
      const int l = w / TE, e = w - l * TE;
      float iv[3] = {0.f, 0.f, 0.f};
      if (e < ne) {
        const float* q = sQ + e * QS + l * 10;
        const float* de = sDraw + e * DS;
        iv[0] = dt * q[6];
        iv[1] = dt * q[7];
        iv[2] = dt * q[8];
        float ci = dt;
#pragma unroll
        for (int o = 1; o <= N; ++o) {
          ci *= dt * (1.f / static_cast<float>(o + 1));
          if (l < n_modes(N - o)) {
            const float* dd = de + d_offset(N, o) + l * 9 + 6;
#pragma unroll
            for (int m = 0; m < 3; ++m) iv[m] = fmaf(ci, dd[m], iv[m]);
          }
        }
      }
#pragma unroll
      for (int ep = 0; ep < 3; ++ep)
#pragma unroll
        for (int m = 0; m < 3; ++m) sM[(ep * L + l) * NM + e * 3 + m] = iv[m];
    }
    // GEMM operand: U(t_z) = sum_o t_z^o / o! D^o at mode l for channels c = eps_xx..eps_zx,
    // alpha, 0.  Lane (c, l mod 4) of a warp holds one channel of one mode for all time
    // nodes, so each store of a warp fills one core matrix without bank conflicts.
    {
      float cf[NT][N];                       // t_z^o / o!, o = 1..N
#pragma unroll
      for (int z = 0; z < NT; ++z) {
        float cc = 1.f;
#pragma unroll
        for (int o = 1; o <= N; ++o) {
          cc *= tz[z] * (1.f / static_cast<float>(o));
          cf[z][o - 1] = cc;
        }
      }
      const int c = lane & 7, l4 = lane >> 3;
      // warps 9..15 and 0 (little or no work above) take the third round of items
      for (int pi = (warp + 7) % 16; pi < TE * (KP / 4); pi += C::THREADS / 32) {
        const int e = pi / (KP / 4), lq = pi - e * (KP / 4);
        const int l = lq * 4 + l4;
        float base = 0.f, dd[N + 1];
#pragma unroll
        for (int o = 0; o <= N; ++o) dd[o] = 0.f;
        if (l < L && e < ne && c < 7) {
          const float* q = sQ + e * QS + l * 10;
          const float* de = sDraw + e * DS;
          base = q[c < 6 ? c : 9];
#pragma unroll
          for (int o = 1; o <= N; ++o) {
            if (c < 6) {
              if (l < n_modes(N - o)) dd[o] = de[d_offset(N, o) + l * 9 + c];
            } else if (o == 1) {
              dd[1] = de[AOFF + l];
            }
          }
        }
#pragma unroll
        for (int z = 0; z < NT; ++z) {
          float x = base;
#pragma unroll
          for (int o = 1; o <= N; ++o) x = fmaf(cf[z][o - 1], dd[o], x);
          const float h = tc::tf32_hi(x);
          const int idx = tc_canon(e * NCOL + z * 8 + c, l, KP);
          sBeH[idx] = h;
          sBeL[idx] = tc::tf32_hi(x - h);
        }
      }
    }
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncthreads();
    if (tid == C::ISSUER) {
      tc::fence_after();
      constexpr uint32_t idesc = tc::idesc_tf32(128, NBC);
      const uint32_t bH = tc::smem_u32(sBeH), bL = tc::smem_u32(sBeL);
#pragma unroll
      for (int ks = 0; ks < KP / 8; ++ks) {
        const uint32_t off = ks * 256;   // 8 K-elements = 2 core matrices
        const uint32_t aH = tmem + C::COL_PH + 8 * ks, aL = tmem + C::COL_PL + 8 * ks;
        tc::mma_tf32_ta(tmem, aH, tc::desc_kmajor(bH + off, KP), idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ta(tmem, aH, tc::desc_kmajor(bL + off, KP), idesc, 1u);
        tc::mma_tf32_ta(tmem, aL, tc::desc_kmajor(bH + off, KP), idesc, 1u);
      }
      tc::commit(&mbar);
    }
    // while the tensor cores run, on the worker warps: the face term (scaled face fluxes,
    // face GEMM), which needs no volume result
    if (tid < C::WORKERS) {
      auto bar = [] { tc::named_barrier(5, C::WORKERS); };
      // one 9-float row (element e, face f, node i) per thread, element fastest: the rows
      // of a warp start 9 floats + a multiple of 36 apart, on distinct banks
      for (int w = tid; w < TE * 4 * NF; w += C::WORKERS) {
        const int e = w % TE, fi = w / TE;
        const int f = fi / NF, i = fi - f * NF;
        float* dst = sF + fi * NFC + e * 9;
        const float sc = e < ne ? sGeo[e * 32 + 17 + f] : 0.f;
        const float* src = sFraw + (e * 4 + f) * FFS + i * 9;
#pragma unroll
        for (int p = 0; p < 9; ++p) dst[p] = e < ne ? sc * src[p] : 0.f;
      }
      bar();
      block_gemm_part<C::KS_FACE, C::NJ_FACE>(sVfw, LP, sF, NFC, LP, NFC, 4 * NF, sPart, [&](int k, int col, float v) {
        if (k < L) {
          const int e = col / 9, p = col - 9 * e;
          sA[(e * L + k) * 10 + p] -= v;
        }
      }, tid, C::WORKERS, bar);
    }
    const bool ok = tc::wait_parity(&mbar, phase, wait_limit);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after();
    // volume nodes: stress and damage rate at the time nodes, time integral; the nodal
    // terms become the projection's B operand (row e*10 + c, column q), split like the
    // volume operand.  Rows [NB, NPC) are zero.
    for (int w = tid; w < (NPC - C::NB) / 8 * C::PGS; w += blockDim.x) {
      sBpH[C::NB / 8 * C::PGS + w] = 0.f;
      sBpL[C::NB / 8 * C::PGS + w] = 0.f;
    }
    {
      const int q = 32 * (warp & 3) + lane;
      const uint32_t lane_base = static_cast<uint32_t>(32 * (warp & 3)) << 16;
#pragma unroll 1
      for (int ei = 0; ei < TE / C::GROUPS; ++ei) {
        const int e = (warp >> 2) * (TE / C::GROUPS) + ei;
        float v[NCOL];
        tc::ld_cols<NCOL>(tmem + lane_base + e * NCOL, v);
        tc::wait_ld();
        float out[10];
#pragma unroll
        for (int c = 0; c < 10; ++c) out[c] = 0.f;
        if (q < NQ && e < ne) {
          const float* gm = sGeo + e * 32;
          MatF m;
          m.rho = gm[9]; m.lam0 = gm[10]; m.mu0 = gm[11]; m.gamma_r = gm[12];
          m.xi0 = gm[13]; m.cd = gm[14]; m.rho_inv = gm[15]; m.pad = 0.f;
          const float* ti = gm;
          float sb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, rb = 0.f;
#pragma unroll
          for (int z = 0; z < NT; ++z) {
            float sig[6], r;
            law_point<LAW>(a.law, v + z * 8, v[z * 8 + 6], m, sig, &r);
#pragma unroll
            for (int p = 0; p < 6; ++p) sb[p] = fmaf(gz[z], sig[p], sb[p]);
            rb = fmaf(gz[z], r, rb);
          }
          const float S[3][3] = {{sb[0], sb[3], sb[5]}, {sb[3], sb[1], sb[4]}, {sb[5], sb[4], sb[2]}};
#pragma unroll
          for (int ep = 0; ep < 3; ++ep)
#pragma unroll
            for (int mc = 0; mc < 3; ++mc)
              out[ep * 3 + mc] =
                  -m.rho_inv * (ti[ep * 3 + 0] * S[mc][0] + ti[ep * 3 + 1] * S[mc][1] + ti[ep * 3 + 2] * S[mc][2]);
          out[9] = rb;
        }
        if (q == 0) {
#pragma unroll
          for (int c = 0; c < 10; ++c) sC[e * 10 + c] = out[c];
        }
        // the terms enter the projection less their value at node 0, which comes back
        // through the row sums of w_q phi_l(x_q): a smooth field keeps its full precision
        tc::named_barrier(1 + (warp >> 2), 128);
        if (q < KQ) {
#pragma unroll
          for (int c = 0; c < 10; ++c) {
            const float x = q < NQ ? out[c] - sC[e * 10 + c] : 0.f;
            const int idx = C::prj_canon(e * 10 + c, q);
            const float h = tc::tf32_hi(x);
            sBpH[idx] = h;
            sBpL[idx] = tc::tf32_hi(x - h);
          }
        }
      }
    }
    // projection on the tensor cores: D[l][n] = sum_q w_q phi_l(x_q) B[n][q], 3xTF32
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncthreads();
    if (tid == C::ISSUER) {
      tc::fence_after();
      constexpr uint32_t idesc = tc::idesc_tf32(128, NPC);
      const uint32_t bH = tc::smem_u32(sBpH), bL = tc::smem_u32(sBpL);
      constexpr uint32_t lbo = 4u * C::PLBO, sbo = 4u * C::PGS;
#pragma unroll
      for (int ks = 0; ks < KQ / 8; ++ks) {
        const uint32_t off = ks * 2 * lbo;   // 8 K-elements = 2 core matrices
        const uint32_t aH = tmem + C::COL_AH + 8 * ks, aL = tmem + C::COL_AL + 8 * ks;
        tc::mma_tf32_ta(tmem + C::COL_DP, aH, tc::desc_kmajor_strided(bH + off, lbo, sbo), idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32_ta(tmem + C::COL_DP, aH, tc::desc_kmajor_strided(bL + off, lbo, sbo), idesc, 1u);
        tc::mma_tf32_ta(tmem + C::COL_DP, aL, tc::desc_kmajor_strided(bH + off, lbo, sbo), idesc, 1u);
      }
      tc::commit(&mbar);
    }
    // while the tensor cores run, on the worker warps: the next tile's copies into the
    // other buffer, the velocity half of the modal derivative, strain rows
    if (tid < C::WORKERS) {
      if (tile + gridDim.x < ntiles)
        issue(tile + gridDim.x, sm + C::oBuf + ((it + 1) & 1) * C::BUF, reinterpret_cast<const int*>(buf + C::bI), tid,
              C::WORKERS);
      modal_derivative_half<N, TE>(sKtB, sM, sH, 0, tid, C::WORKERS);
      tc::named_barrier(5, C::WORKERS);
      strain_rows<N, TE>(sH, sGeo, sA, tid, C::WORKERS);
    }
    tc::cp_async_commit();
    {
      const bool ok2 = tc::wait_parity(&mbar, phase, wait_limit);
      phase ^= 1u;
      if (__syncthreads_or(!ok2)) {
        failed = true;
        break;
      }
    }
    tc::fence_after();
    // read-out: warps 0, 1 of group g hold modes [0, 64) of element g
    if ((warp & 3) < 2) {
      const int l = 32 * (warp & 3) + lane, e = warp >> 2;
      float v[40];
      tc::ld_cols<40>(tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + C::COL_DP, v);
      tc::wait_ld();
      if (l < L) {
        const float sl = __ldg(tb + T.PrjS + l);
        const float* ce = sC + e * 10;
#pragma unroll
        for (int ee = 0; ee < TE; ++ee) {
          if (ee == e) {
#pragma unroll
            for (int c = 0; c < 9; ++c) sM[((c / 3) * L + l) * NM + NV + ee * 3 + c % 3] = fmaf(ce[c], sl, v[ee * 10 + c]);
            sA[(ee * L + l) * 10 + 9] += fmaf(ce[9], sl, v[ee * 10 + 9]);
          }
        }
      }
    }
    tc::fence_before();
    __syncthreads();
    modal_derivative_half<N, TE>(sKtB, sM, sH, NV, tid, blockDim.x);
    __syncthreads();
    velocity_rows<N, TE>(sH, sA);
    __syncthreads();
    // update
    bool bad = false;
    for (int w = tid; w < ne * L * 10; w += blockDim.x) {
      const int e = w / (L * 10), r = w - e * (L * 10);
      const float v = sQ[e * QS + r] + sA[e * L * 10 + r];
      bad |= !isfinite(v);
      a.q_out[(e0 + e) * QS + r] = v;
    }
    if (bad) atomicOr(a.status, kStatusNonFinite);
  }
  tc::cp_async_wait<0>();                    // no copy may still be in flight at exit
  if (failed) {
    if (tid == 0) atomicOr(a.status, kStatusTimeout);
    tc::wait_parity(&mbar, phase ^ 1u, kWaitLimit);   // let the MMAs in flight finish before freeing TMEM
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, C::TMEM_COLS);
}

// ---------------------------------------------------------------------------
template <class Cfg, class Kern>
cudaError_t launch_persistent(Kern kern, int64_t tiles, int grid_hint, const StepArgs& a, cudaStream_t s,
                              bool* configured, int* max_blocks, int cap_per_sm = 0) {
  const size_t smem = sizeof(float) * Cfg::SMEM;
  if (!*configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cap_per_sm > 0) {
      // Kernels holding tensor memory: the occupancy query counts one block per SM for any
      // kernel that allocates it, whatever it allocates.  The blocks that shared memory,
      // registers and threads allow are resident; of those, cap_per_sm fit in the SM's
      // 512 columns (a block that finds too few waits in its allocation, it cannot deadlock).
      cudaFuncAttributes fa{};
      e = cudaFuncGetAttributes(&fa, kern);
      if (e != cudaSuccess) return e;
      int dev = 0, sm_smem = 0, reserved = 0, sm_regs = 0, sm_threads = 0;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
          (e = cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
        return e;
      const int warps = (Cfg::THREADS + 31) / 32;
      const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;      // allocated per warp in units of 256
      const int by_smem = static_cast<int>(static_cast<size_t>(sm_smem) / (smem + fa.sharedSizeBytes + reserved));
      const int by_regs = regs_warp > 0 ? sm_regs / (regs_warp * warps) : cap_per_sm;
      const int by_threads = sm_threads / Cfg::THREADS;
      per_sm = std::min(std::min(by_smem, by_regs), std::min(by_threads, cap_per_sm));
    } else {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::THREADS, smem);
      if (e != cudaSuccess) return e;
    }
    *max_blocks = per_sm > 0 ? per_sm : 1;
    *configured = true;
  }
  int64_t grid = grid_hint > 0 ? static_cast<int64_t>(grid_hint) * *max_blocks : tiles;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  kern<<<static_cast<unsigned>(grid), Cfg::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

// Kernel variants (bit 0: predictor with shared-memory tables on a persistent
// grid; bit 2: SIMT corrector likewise; bit 3: SIMT corrector instead of the
// tensor-core one; bit 4: SIMT Picard predictor instead of the tensor-core one;
// bit 5: SIMT predictor instead of the tensor-core one).  Clear bits read the tables
// through the L1 cache with one CTA per tile.  The default is the fastest
// measured combination on GB300; DG_KERNEL_VARIANT overrides it for tuning.
inline int table_residency_mask() {
  static int mask = -1;
  if (mask < 0) {
    const char* s = getenv("DG_KERNEL_VARIANT");
    mask = s ? atoi(s) : 1;
  }
  return mask;
}

template <int N, int LAW>
cudaError_t launch_predictor_law(const StepArgs& a, cudaStream_t s) {
  static bool cfg[3] = {false, false, false};
  static int blocks[3] = {1, 1, 1};
  if constexpr (tc_volume(N)) {
    if (!(table_residency_mask() & 32)) {
      const int64_t tiles = (a.E + PredTcCfg<N>::TE - 1) / PredTcCfg<N>::TE;
      // resident CTAs of an SM share its 512 tensor-memory columns
      return launch_persistent<PredTcCfg<N>>(k_predictor_tc<N, LAW>, tiles, a.grid_pred > 0 ? a.grid_pred : 148, a,
                                             s, &cfg[2], &blocks[2], 512 / PredTcCfg<N>::TMEM_COLS);
    }
  }
  const int64_t tiles = (a.E + PredCfg<N, true>::TE - 1) / PredCfg<N, true>::TE;
  if constexpr (PredCfg<N, true>::FITS) {
    if (table_residency_mask() & 1)
      return launch_persistent<PredCfg<N, true>>(k_predictor<N, true, LAW>, tiles, a.grid_pred, a, s, &cfg[1],
                                                 &blocks[1]);
  }
  return launch_persistent<PredCfg<N, false>>(k_predictor<N, false, LAW>, tiles, 0, a, s, &cfg[0], &blocks[0]);
}

template <int N, int LAW>
cudaError_t launch_faces_law(const StepArgs& a, cudaStream_t s) {
  static bool cfg[2] = {false, false};
  static int blocks[2] = {1, 1};
  const int64_t tiles = (a.F + FluxCfg<N>::TF - 1) / FluxCfg<N>::TF;
  const int grid = a.grid_face > 0 ? a.grid_face : 148;
  if (a.has_boundary)
    return launch_persistent<FluxCfg<N>>(k_face_flux<N, LAW, true>, tiles, grid, a, s, &cfg[1], &blocks[1]);
  return launch_persistent<FluxCfg<N>>(k_face_flux<N, LAW, false>, tiles, grid, a, s, &cfg[0], &blocks[0]);
}

template <int N, int LAW>
cudaError_t launch_corrector_law(const StepArgs& a, cudaStream_t s) {
  static bool cfg[3] = {false, false, false};
  static int blocks[3] = {1, 1, 1};
  if constexpr (tc_volume(N)) {
    if (!(table_residency_mask() & 8)) {
      const int64_t tiles = (a.E + CorrTcCfg<N>::TE - 1) / CorrTcCfg<N>::TE;
      // resident CTAs of an SM share its 512 tensor-memory columns
      return launch_persistent<CorrTcCfg<N>>(k_corrector_tc<N, LAW>, tiles, a.grid_corr > 0 ? a.grid_corr : 148, a,
                                             s, &cfg[2], &blocks[2], 512 / CorrTcCfg<N>::TMEM_COLS);
    }
  }
  const int64_t tiles = (a.E + CorrCfg<N, true>::TE - 1) / CorrCfg<N, true>::TE;
  if constexpr (CorrCfg<N, true>::FITS) {
    if (table_residency_mask() & 4)
      return launch_persistent<CorrCfg<N, true>>(k_corrector<N, true, LAW>, tiles, a.grid_corr, a, s, &cfg[1],
                                                 &blocks[1]);
  }
  return launch_persistent<CorrCfg<N, false>>(k_corrector<N, false, LAW>, tiles, 0, a, s, &cfg[0], &blocks[0]);
}

template <int N, int LAW>
cudaError_t launch_picard_law(const StepArgs& a, cudaStream_t s) {
  static bool cfg[2] = {false, false};
  static int blocks[2] = {1, 1};
  if constexpr (tc_volume(N)) {
    if (!(table_residency_mask() & 16)) {
      const int64_t tiles = (a.E + PicTcCfg<N>::TE - 1) / PicTcCfg<N>::TE;
      // resident CTAs of an SM share its 512 tensor-memory columns
      return launch_persistent<PicTcCfg<N>>(k_picard_tc<N, LAW>, tiles, a.grid_corr > 0 ? a.grid_corr : 148, a, s,
                                            &cfg[1], &blocks[1], 512 / PicTcCfg<N>::TMEM_COLS);
    }
  }
  const int64_t tiles = (a.E + PicardCfg<N>::TE - 1) / PicardCfg<N>::TE;
  return launch_persistent<PicardCfg<N>>(k_picard<N, LAW>, tiles, 148, a, s, &cfg[0], &blocks[0]);
}

// The CDM runs on kernels compiled for it alone; the other laws on the dispatching ones.
template <int N>
cudaError_t launch_predictor_impl(const StepArgs& a, cudaStream_t s) {
  return a.law == 0 ? launch_predictor_law<N, 0>(a, s) : launch_predictor_law<N, -1>(a, s);
}
template <int N>
cudaError_t launch_faces_impl(const StepArgs& a, cudaStream_t s) {
  return a.law == 0 ? launch_faces_law<N, 0>(a, s) : launch_faces_law<N, -1>(a, s);
}
template <int N>
cudaError_t launch_corrector_impl(const StepArgs& a, cudaStream_t s) {
  return a.law == 0 ? launch_corrector_law<N, 0>(a, s) : launch_corrector_law<N, -1>(a, s);
}
template <int N>
cudaError_t launch_picard_impl(const StepArgs& a, cudaStream_t s) {
  if constexpr (PicardCfg<N>::FITS)
    return a.law == 0 ? launch_picard_law<N, 0>(a, s) : launch_picard_law<N, -1>(a, s);
  return cudaErrorNotSupported;
}

}  // namespace dg

#define DG_INSTANTIATE_STEP(N)                                                                  \
  namespace dg {                                                                                \
  template <> cudaError_t launch_predictor_t<N>(const StepArgs& a, cudaStream_t s) {           \
    return launch_predictor_impl<N>(a, s);                                                      \
  }                                                                                             \
  template <> cudaError_t launch_faces_t<N>(const StepArgs& a, cudaStream_t s) {               \
    return launch_faces_impl<N>(a, s);                                                          \
  }                                                                                             \
  template <> cudaError_t launch_corrector_t<N>(const StepArgs& a, cudaStream_t s) {           \
    return launch_corrector_impl<N>(a, s);                                                      \
  }                                                                                             \
  template <> cudaError_t launch_picard_t<N>(const StepArgs& a, cudaStream_t s) {              \
    return launch_picard_impl<N>(a, s);                                                         \
  }                                                                                             \
  }
