// Predictor and corrector kernels of one ADER-DG step for the CDM damage
// rheology (arXiv 2502.09714, Appendix A), FP32, templated on the degree N.
//
// Data per element (see dg_internal.h): modal state Q[L][10]; predictor output
// D^i (i = 1..N) of the 9 wave fields on the modes of degree <= N-i, plus
// D^1 of alpha on all modes.  A CTA processes TE consecutive elements; their
// data is staged in shared memory and the reference tables are read through
// the read-only cache.
#pragma once

#include "dg_internal.h"

namespace dg {

template <int N>
struct Dims {
  static constexpr int L = n_modes(N);
  static constexpr int NQ = n_vol_nodes(N);
  static constexpr int NF = n_face_nodes(N);
  static constexpr int NT = N + 1;
  static constexpr int QS = q_stride(N);
  static constexpr int DS = d_stride(N);
  static constexpr int AOFF = d_alpha_offset(N);
  // elements per CTA
  static constexpr int TE = N <= 2 ? 16 : (N == 3 ? 8 : 4);
  // corrector scratch per element: volume-node data or neighbour copies + face fluxes
  static constexpr int XS_VOL = NQ * 10;
  static constexpr int XS_FACE = QS + DS + NF * 9;
  static constexpr int XS = round4(XS_VOL > XS_FACE ? XS_VOL : XS_FACE);
  static constexpr int IS = round4(L * 3);
  static constexpr int AS = round4(L * 10);
  static constexpr int PRED_SMEM = TE * (QS + 2 * round4(L * 9) + round4(NQ) + 16);
  static constexpr int CORR_SMEM = TE * (QS + DS + AS + IS + XS);
};

__host__ __device__ constexpr int lr(int N, int i) { return n_modes(N - i); }

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

// Normal flux F^d(u) n_d of the 9 wave fields (Eq. "nonlinear hyper pdes"):
// strain rows -(v_i n_j + v_j n_i)/2, velocity rows -sigma_ij n_j / rho.
__device__ __forceinline__ void normal_flux(const float u[10], const MatF& m, const float n[3], float F[9]) {
  float sig[6], r;
  cdm_point(u, u[9], m, sig, &r);
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

// ---------------------------------------------------------------------------
// Predictor: cell-mean effective Jacobian, Cauchy-Kovalevskaya recursion
// (Eq. "CKIter-ref-matrix") and the damage-rate source at i = 1
// (Eq. "CKIter-ref-source").
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_predictor(StepArgs a) {
  using Dm = Dims<N>;
  constexpr int L = Dm::L, NQ = Dm::NQ, QS = Dm::QS, DS = Dm::DS, TE = Dm::TE;
  constexpr int L9 = round4(L * 9);
  constexpr TableLayout T = table_layout(N);
  extern __shared__ float4 smem4[];
  float* sQ = reinterpret_cast<float*>(smem4);   // [TE][QS]
  float* sP = sQ + TE * QS;                      // [TE][L9] D^i for odd i
  float* sN = sP + TE * L9;                      // [TE][L9] D^i for even i
  float* sR = sN + TE * L9;                      // [TE][NQ] damage rate at the nodes
  float* sC = sR + TE * round4(NQ);              // [TE][16] per-element coefficients
  const float* tb = a.tables;
  const int64_t e0 = static_cast<int64_t>(blockIdx.x) * TE;
  const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));

  {
    const float4* src = reinterpret_cast<const float4*>(a.q_in + e0 * QS);
    float4* dst = reinterpret_cast<float4*>(sQ);
    for (int w = threadIdx.x; w < ne * QS / 4; w += blockDim.x) dst[w] = __ldg(src + w);
  }
  __syncthreads();

  if (threadIdx.x < ne) {
    const int e = threadIdx.x;
    const int64_t ge = e0 + e;
    const MatF m = a.mat[ge];
    const float r6 = 2.449489742783178f;   // phi_0 = sqrt(6): cell mean = Q_0 sqrt(6)
    float u[6];
    for (int p = 0; p < 6; ++p) u[p] = sQ[e * QS + p] * r6;
    const float alpha = sQ[e * QS + 9] * r6;
    const float I1 = u[0] + u[1] + u[2];
    const float I2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + 2.f * (u[3] * u[3] + u[4] * u[4] + u[5] * u[5]);
    const float xi = I2 > 1e-30f ? I1 * rsqrtf(I2) : 0.f;
    // effective Lame parameters at the cell mean (Eq. "effective-cdb", mu sign from Eq. "cdb-model")
    const float lam = m.lam0 - alpha * m.gamma_r * xi * (1.f / 3.f);
    const float mu = m.mu0 + alpha * m.xi0 * m.gamma_r - 0.5f * alpha * m.gamma_r * xi;
    if (!(mu > 0.f) || !(lam + 2.f * mu > 0.f)) atomicOr(a.status, kStatusNonHyperbolic);
    a.cp[ge] = sqrtf(fmaxf(lam + 2.f * mu, 0.f) * m.rho_inv);
    float* c = sC + e * 16;
    c[0] = lam * m.rho_inv;
    c[1] = mu * m.rho_inv;
    const GeomF* g = a.geom + ge;
    for (int k = 0; k < 9; ++k) c[2 + k] = g->tinv[k];
  }

  // damage rate at the volume nodes from the state at t_n
  for (int w = threadIdx.x; w < ne * NQ; w += blockDim.x) {
    const int e = w / NQ, q = w - e * NQ;
    const float* vv = tb + T.Vv + q * L;
    const float* qe = sQ + e * QS;
    float eps[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int l = 0; l < L; ++l) {
      const float phi = __ldg(vv + l);
#pragma unroll
      for (int p = 0; p < 6; ++p) eps[p] = fmaf(phi, qe[l * 10 + p], eps[p]);
    }
    sR[e * round4(NQ) + q] = cdm_rate(eps, a.mat[e0 + e]);
  }
  __syncthreads();
  // D^1 of alpha = projection of the rate (mass matrix = identity)
  for (int w = threadIdx.x; w < ne * L; w += blockDim.x) {
    const int e = w / L, k = w - e * L;
    const float* r = sR + e * round4(NQ);
    float acc = 0.f;
    for (int q = 0; q < NQ; ++q) acc = fmaf(__ldg(tb + T.Vw + q * L + k), r[q], acc);
    a.d[(e0 + e) * DS + Dm::AOFF + k] = acc;
  }

  // Cauchy-Kovalevskaya: D^i_kp = -sum_e Kt^e_kl D^{i-1}_lq (Theta^{-1}_ed B^d_pq)
#pragma unroll 1
  for (int i = 1; i <= N; ++i) {
    const int Lin = n_modes(N - i + 1), Lout = n_modes(N - i);
    const float* prev = (i == 1) ? sQ : ((i & 1) ? sN : sP);
    const int pstride = (i == 1) ? QS : L9;
    const int pld = (i == 1) ? 10 : 9;
    float* cur = (i & 1) ? sP : sN;
    const int doff = d_offset(N, i);
    for (int w = threadIdx.x; w < ne * Lout; w += blockDim.x) {
      const int e = w / Lout, k = w - e * Lout;
      float g[3][9];
#pragma unroll
      for (int f = 0; f < 9; ++f) g[0][f] = g[1][f] = g[2][f] = 0.f;
      const float* kt = tb + T.Kt + k * L;
      const float* pe = prev + e * pstride;
      for (int l = 0; l < Lin; ++l) {
        const float k0 = __ldg(kt + l), k1 = __ldg(kt + L * L + l), k2 = __ldg(kt + 2 * L * L + l);
        const float* pr = pe + l * pld;
#pragma unroll
        for (int f = 0; f < 9; ++f) {
          const float v = pr[f];
          g[0][f] = fmaf(k0, v, g[0][f]);
          g[1][f] = fmaf(k1, v, g[1][f]);
          g[2][f] = fmaf(k2, v, g[2][f]);
        }
      }
      const float* c = sC + e * 16;
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
      float* out = cur + e * L9 + k * 9;
      float* gout = a.d + (e0 + e) * DS + doff + k * 9;
#pragma unroll
      for (int f = 0; f < 9; ++f) {
        out[f] = Di[f];
        gout[f] = Di[f];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Corrector: volume flux and damage source by space-time quadrature
// (Eqs. "3rd term", "rhs term"), Rusanov face flux with the neighbour trace
// (Eqs. "rusanov-flux", "2nd term"), update (Eq. "time-integrated").
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_corrector(StepArgs a) {
  using Dm = Dims<N>;
  constexpr int L = Dm::L, NQ = Dm::NQ, NF = Dm::NF, NT = Dm::NT, QS = Dm::QS, DS = Dm::DS;
  constexpr int TE = Dm::TE, XS = Dm::XS, IS = Dm::IS, AS = Dm::AS, AOFF = Dm::AOFF;
  constexpr TableLayout T = table_layout(N);
  extern __shared__ float4 smem4[];
  float* sQ = reinterpret_cast<float*>(smem4);   // [TE][QS]  own state
  float* sD = sQ + TE * QS;                      // [TE][DS]  own predictor
  float* sA = sD + TE * DS;                      // [TE][AS]  update accumulator
  float* sI = sA + TE * AS;                      // [TE][IS]  time-integrated velocity
  float* sX = sI + TE * IS;                      // [TE][XS]  scratch
  const float* tb = a.tables;
  const float dt = a.dt;
  const int64_t e0 = static_cast<int64_t>(blockIdx.x) * TE;
  const int ne = static_cast<int>(min(static_cast<int64_t>(TE), a.E - e0));

  {
    const float4* srcq = reinterpret_cast<const float4*>(a.q_in + e0 * QS);
    const float4* srcd = reinterpret_cast<const float4*>(a.d + e0 * DS);
    for (int w = threadIdx.x; w < ne * QS / 4; w += blockDim.x) reinterpret_cast<float4*>(sQ)[w] = __ldg(srcq + w);
    for (int w = threadIdx.x; w < ne * DS / 4; w += blockDim.x) reinterpret_cast<float4*>(sD)[w] = __ldg(srcd + w);
    for (int w = threadIdx.x; w < TE * AS; w += blockDim.x) sA[w] = 0.f;
  }
  __syncthreads();

  // time integral of the velocity Taylor series over [0, dt]
  for (int w = threadIdx.x; w < ne * L; w += blockDim.x) {
    const int e = w / L, l = w - e * L;
    float iv[3];
    for (int m = 0; m < 3; ++m) iv[m] = dt * sQ[e * QS + l * 10 + 6 + m];
    float c = dt;
#pragma unroll
    for (int o = 1; o <= N; ++o) {
      c *= dt / static_cast<float>(o + 1);
      if (l < n_modes(N - o))
        for (int m = 0; m < 3; ++m) iv[m] = fmaf(c, sD[e * DS + d_offset(N, o) + l * 9 + 6 + m], iv[m]);
    }
    for (int m = 0; m < 3; ++m) sI[e * IS + l * 3 + m] = iv[m];
  }

  // volume nodes: strain and damage in time, CDM stress and rate, time integral
  for (int w = threadIdx.x; w < ne * NQ; w += blockDim.x) {
    const int e = w / NQ, q = w - e * NQ;
    const int64_t ge = e0 + e;
    const MatF m = a.mat[ge];
    const float* vv = tb + T.Vv + q * L;
    const float* qe = sQ + e * QS;
    const float* de = sD + e * DS;
    float t0[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float ta1 = 0.f;
    for (int l = 0; l < L; ++l) {
      const float phi = __ldg(vv + l);
#pragma unroll
      for (int p = 0; p < 6; ++p) t0[p] = fmaf(phi, qe[l * 10 + p], t0[p]);
      t0[6] = fmaf(phi, qe[l * 10 + 9], t0[6]);
      ta1 = fmaf(phi, de[AOFF + l], ta1);
    }
    float th[N][6];
#pragma unroll
    for (int o = 1; o <= N; ++o) {
#pragma unroll
      for (int p = 0; p < 6; ++p) th[o - 1][p] = 0.f;
      const float* dd = de + d_offset(N, o);
      for (int l = 0; l < n_modes(N - o); ++l) {
        const float phi = __ldg(vv + l);
#pragma unroll
        for (int p = 0; p < 6; ++p) th[o - 1][p] = fmaf(phi, dd[l * 9 + p], th[o - 1][p]);
      }
    }
    float sb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, rb = 0.f;
#pragma unroll
    for (int z = 0; z < NT; ++z) {
      const float tau = __ldg(tb + T.tz + z) * dt, gam = __ldg(tb + T.gz + z) * dt;
      float eps[6];
#pragma unroll
      for (int p = 0; p < 6; ++p) eps[p] = t0[p];
      float c = 1.f;
#pragma unroll
      for (int o = 1; o <= N; ++o) {
        c *= tau / static_cast<float>(o);
#pragma unroll
        for (int p = 0; p < 6; ++p) eps[p] = fmaf(c, th[o - 1][p], eps[p]);
      }
      const float alpha = fmaf(tau, ta1, t0[6]);
      float sig[6], r;
      cdm_point(eps, alpha, m, sig, &r);
#pragma unroll
      for (int p = 0; p < 6; ++p) sb[p] = fmaf(gam, sig[p], sb[p]);
      rb = fmaf(gam, r, rb);
    }
    // T[e'][m] = -(1/rho) sum_d Theta^{-1}_{e'd} sigma_md, so that the velocity rows of
    // the volume term are sum_q sum_e' (w_q d phi_k / d xi_e')(x_q) T[e'][m](x_q)
    const float S[3][3] = {{sb[0], sb[3], sb[5]}, {sb[3], sb[1], sb[4]}, {sb[5], sb[4], sb[2]}};
    const float* ti = a.geom[ge].tinv;
    float* x = sX + e * XS + q * 10;
#pragma unroll
    for (int ep = 0; ep < 3; ++ep)
#pragma unroll
      for (int mc = 0; mc < 3; ++mc)
        x[ep * 3 + mc] = -m.rho_inv * (ti[ep * 3 + 0] * S[mc][0] + ti[ep * 3 + 1] * S[mc][1] + ti[ep * 3 + 2] * S[mc][2]);
    x[9] = rb;
  }
  __syncthreads();

  // projections of the volume terms onto the modes
  for (int w = threadIdx.x; w < ne * L; w += blockDim.x) {
    const int e = w / L, k = w - e * L;
    const float* xe = sX + e * XS;
    float acc[3] = {0.f, 0.f, 0.f}, src = 0.f;
    for (int q = 0; q < NQ; ++q) {
      const float* x = xe + q * 10;
      const float g0 = __ldg(tb + T.Gw + (0 * NQ + q) * L + k);
      const float g1 = __ldg(tb + T.Gw + (1 * NQ + q) * L + k);
      const float g2 = __ldg(tb + T.Gw + (2 * NQ + q) * L + k);
#pragma unroll
      for (int mc = 0; mc < 3; ++mc) acc[mc] += g0 * x[mc] + g1 * x[3 + mc] + g2 * x[6 + mc];
      src = fmaf(__ldg(tb + T.Vw + q * L + k), x[9], src);
    }
    // strain rows (linear in v): -(1/2) int (v_i d_j phi_k + v_j d_i phi_k), taken modally
    float H[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    const float* iv = sI + e * IS;
    for (int l = 0; l < L; ++l) {
      const float k0 = __ldg(tb + T.Kt + (0 * L + l) * L + k);
      const float k1 = __ldg(tb + T.Kt + (1 * L + l) * L + k);
      const float k2 = __ldg(tb + T.Kt + (2 * L + l) * L + k);
#pragma unroll
      for (int mc = 0; mc < 3; ++mc) {
        const float v = iv[l * 3 + mc];
        H[0][mc] = fmaf(k0, v, H[0][mc]);
        H[1][mc] = fmaf(k1, v, H[1][mc]);
        H[2][mc] = fmaf(k2, v, H[2][mc]);
      }
    }
    const float* ti = a.geom[e0 + e].tinv;
    float hd[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int mc = 0; mc < 3; ++mc) hd[d][mc] = ti[0 * 3 + d] * H[0][mc] + ti[1 * 3 + d] * H[1][mc] + ti[2 * 3 + d] * H[2][mc];
    float* acc_out = sA + e * AS + k * 10;
    acc_out[0] -= hd[0][0];
    acc_out[1] -= hd[1][1];
    acc_out[2] -= hd[2][2];
    acc_out[3] -= 0.5f * (hd[1][0] + hd[0][1]);
    acc_out[4] -= 0.5f * (hd[2][1] + hd[1][2]);
    acc_out[5] -= 0.5f * (hd[0][2] + hd[2][0]);
    acc_out[6] += acc[0];
    acc_out[7] += acc[1];
    acc_out[8] += acc[2];
    acc_out[9] += src;
  }
  __syncthreads();

  // faces
#pragma unroll 1
  for (int f = 0; f < 4; ++f) {
    // stage the neighbours' state and predictor
    constexpr int CH = (QS + DS) / 4;
    for (int w = threadIdx.x; w < ne * CH; w += blockDim.x) {
      const int e = w / CH, c = w - e * CH;
      const int nbv = a.nbr[(e0 + e) * 4 + f];
      const int64_t nbe = nbv >> 2;
      float4 v;
      if (c < QS / 4) v = __ldg(reinterpret_cast<const float4*>(a.q_in + nbe * QS) + c);
      else v = __ldg(reinterpret_cast<const float4*>(a.d + nbe * DS) + (c - QS / 4));
      reinterpret_cast<float4*>(sX + e * XS)[c] = v;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ne * NF; w += blockDim.x) {
      const int e = w / NF, i = w - e * NF;
      const int64_t ge = e0 + e;
      const int nbv = a.nbr[ge * 4 + f];
      const int64_t nbe = nbv >> 2;
      const int fn = nbv & 3;
      const float* vo = tb + T.Vf + (f * NF + i) * L;
      const float* vn = tb + T.Vf + (fn * NF + i) * L;
      const float* qo = sQ + e * QS;
      const float* dO = sD + e * DS;
      const float* qn = sX + e * XS;
      const float* dn = qn + QS;
      float o0[10], n0[10], oa1 = 0.f, na1 = 0.f;
#pragma unroll
      for (int p = 0; p < 10; ++p) o0[p] = n0[p] = 0.f;
      for (int l = 0; l < L; ++l) {
        const float po = __ldg(vo + l), pn = __ldg(vn + l);
#pragma unroll
        for (int p = 0; p < 10; ++p) {
          o0[p] = fmaf(po, qo[l * 10 + p], o0[p]);
          n0[p] = fmaf(pn, qn[l * 10 + p], n0[p]);
        }
        oa1 = fmaf(po, dO[AOFF + l], oa1);
        na1 = fmaf(pn, dn[AOFF + l], na1);
      }
      float oh[N][9], nh[N][9];
#pragma unroll
      for (int o = 1; o <= N; ++o) {
#pragma unroll
        for (int p = 0; p < 9; ++p) oh[o - 1][p] = nh[o - 1][p] = 0.f;
        const int off = d_offset(N, o);
        for (int l = 0; l < n_modes(N - o); ++l) {
          const float po = __ldg(vo + l), pn = __ldg(vn + l);
#pragma unroll
          for (int p = 0; p < 9; ++p) {
            oh[o - 1][p] = fmaf(po, dO[off + l * 9 + p], oh[o - 1][p]);
            nh[o - 1][p] = fmaf(pn, dn[off + l * 9 + p], nh[o - 1][p]);
          }
        }
      }
      const GeomF* g = a.geom + ge;
      const float n[3] = {g->face[f][0], g->face[f][1], g->face[f][2]};
      const float scale = g->face[f][3];
      const MatF mo = a.mat[ge], mn = a.mat[nbe];
      const float C = fmaxf(a.cp[ge], a.cp[nbe]);
      float Fb[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) Fb[p] = 0.f;
#pragma unroll
      for (int z = 0; z < NT; ++z) {
        const float tau = __ldg(tb + T.tz + z) * dt, gam = __ldg(tb + T.gz + z) * dt;
        float um[10], up[10];
#pragma unroll
        for (int p = 0; p < 10; ++p) { um[p] = o0[p]; up[p] = n0[p]; }
        um[9] = fmaf(tau, oa1, um[9]);
        up[9] = fmaf(tau, na1, up[9]);
        float c = 1.f;
#pragma unroll
        for (int o = 1; o <= N; ++o) {
          c *= tau / static_cast<float>(o);
#pragma unroll
          for (int p = 0; p < 9; ++p) {
            um[p] = fmaf(c, oh[o - 1][p], um[p]);
            up[p] = fmaf(c, nh[o - 1][p], up[p]);
          }
        }
        float Fm[9], Fp[9];
        normal_flux(um, mo, n, Fm);
        normal_flux(up, mn, n, Fp);
#pragma unroll
        for (int p = 0; p < 9; ++p) Fb[p] = fmaf(gam, 0.5f * (Fm[p] + Fp[p]) + 0.5f * C * (um[p] - up[p]), Fb[p]);
      }
      float* fo = sX + e * XS + QS + DS + i * 9;
#pragma unroll
      for (int p = 0; p < 9; ++p) fo[p] = Fb[p] * scale;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ne * L; w += blockDim.x) {
      const int e = w / L, k = w - e * L;
      const float* fe = sX + e * XS + QS + DS;
      float acc[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) acc[p] = 0.f;
      for (int i = 0; i < NF; ++i) {
        const float v = __ldg(tb + T.Vfw + (f * NF + i) * L + k);
#pragma unroll
        for (int p = 0; p < 9; ++p) acc[p] = fmaf(v, fe[i * 9 + p], acc[p]);
      }
      float* ao = sA + e * AS + k * 10;
#pragma unroll
      for (int p = 0; p < 9; ++p) ao[p] -= acc[p];
    }
    __syncthreads();
  }

  // update
  bool bad = false;
  for (int w = threadIdx.x; w < ne * L * 10; w += blockDim.x) {
    const int e = w / (L * 10), r = w - e * (L * 10);
    const float v = sQ[e * QS + r] + sA[e * AS + r];
    bad |= !isfinite(v);
    a.q_out[(e0 + e) * QS + r] = v;
  }
  if (bad) atomicOr(a.status, kStatusNonFinite);
}

template <int N>
cudaError_t launch_predictor_impl(const StepArgs& a, cudaStream_t s) {
  using Dm = Dims<N>;
  const size_t smem = sizeof(float) * Dm::PRED_SMEM;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t blocks = (a.E + Dm::TE - 1) / Dm::TE;
  k_predictor<N><<<static_cast<unsigned>(blocks), 128, smem, s>>>(a);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_corrector_impl(const StepArgs& a, cudaStream_t s) {
  using Dm = Dims<N>;
  const size_t smem = sizeof(float) * Dm::CORR_SMEM;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_corrector<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t blocks = (a.E + Dm::TE - 1) / Dm::TE;
  k_corrector<N><<<static_cast<unsigned>(blocks), 128, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dg

#define DG_INSTANTIATE_STEP(N)                                                                  \
  namespace dg {                                                                                \
  template <> cudaError_t launch_predictor_t<N>(const StepArgs& a, cudaStream_t s) {           \
    return launch_predictor_impl<N>(a, s);                                                      \
  }                                                                                             \
  template <> cudaError_t launch_corrector_t<N>(const StepArgs& a, cudaStream_t s) {           \
    return launch_corrector_impl<N>(a, s);                                                      \
  }                                                                                             \
  }
