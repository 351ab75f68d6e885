// Discrete adjoint of one CK step under the CDM law (Eq. "cdb-model"), FP32,
// templated on the degree N.  With lam = dJ/dQ^{k+1}, the two kernels give
// dJ/dQ^k and add dJ/dxi0 and dJ/dC_d of the step
//     Q^{k+1} = Q^k + vol(U) + src(U) - face(U, U_nbr, C) / |J|
// (Eqs. "time-integrated", "3rd term", "rhs term", "2nd term", "rusanov-flux";
// U the Taylor expansion of the CK predictor, Eqs. "CKIter-ref-matrix" and
// "CKIter-ref-source"), every product of the forward step transposed:
//
//   k_adj_face   once per face: lam of the face term -> lam of both traces at
//                the space-time face nodes through the Rusanov flux (flux
//                Jacobians of both sides, C = max of the two P speeds), folded
//                into Taylor orders and projected onto the modes of each side;
//                lam of C and the xi0 part per side.  A free-surface or
//                absorbing face transposes its boundary flux (Appendix A) and
//                returns the flux's derivatives in the own cell's effective
//                Lame parameters.
//   k_adj_elem   once per element: volume flux and damage-rate source
//                transposed at the space-time volume nodes, the records of its
//                four faces gathered, the CK recursion transposed from order N
//                down to 0 (star matrices through the effective Lame
//                parameters of the cell mean, damage-rate source of D^1), and
//                the cell-mean terms; writes dJ/dQ^k = lam + dJ/dD^0 and adds
//                the element's parameter gradient in FP64.
//
// Conventions at the non-smooth points: the damage rate has derivative zero
// where I1 sqrt(I2) - xi0 I2 <= 0, xi and sqrt(I2) have derivative zero below
// I2 = 1e-30, and a tie of the two P speeds splits the derivative of the max in
// halves.  The predictor output D and the speeds cp of Q^k come from the
// forward predictor kernel, launched on Q^k just before.
#pragma once

#include "dg_internal.h"
#include "dg_tc.cuh"

namespace dg {
namespace adj {

template <int N>
struct ADim {
  static constexpr int L = n_modes(N), NQ = n_vol_nodes(N), NF = n_face_nodes(N), NT = N + 1;
  static constexpr int LP = lp_of(N), NQP = nqp_of(N), NFP = nfp_of(N);
  static constexpr int QS = q_stride(N), DS = d_stride(N), AOFF = d_alpha_offset(N);
  static constexpr int RS = adj_rec_stride(N);
  static constexpr int LDS = QS + DS;           // lam of D^0..D^N in the (Q, D) layout
  static constexpr int U0S = NQP + 4;           // row stride of the nodal lam of the damage source (off the bank period)
  // rows (i, k), k < L_{N-i}, of the forward CK products of the transposed recursion
  __host__ __device__ static constexpr int gx_row(int i) {
    int r = 0;
    for (int j = 1; j < i; ++j) r += n_modes(N - j);
    return r;
  }
  static constexpr int GXI = gx_row(N + 1);
  static_assert(GXI * 27 <= NQ * 28, "forward CK products fit in the X region");
};

// sqrt(I2), xi = I1 / sqrt(I2) and their derivatives in the six strain entries
// (zero below I2 = 1e-30); dI2 counts each shear entry twice.
struct Inv {
  float I1, I2, s, xi, ds[6], dxi[6];
};
__device__ __forceinline__ Inv invariants(const float* e) {
  Inv v;
  v.I1 = e[0] + e[1] + e[2];
  v.I2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + 2.f * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
  if (v.I2 > 1e-30f) {
    const float rs = rsqrtf(v.I2);
    v.s = v.I2 * rs;
    v.xi = v.I1 * rs;
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      v.ds[p] = (p < 3 ? 1.f : 2.f) * e[p] * rs;        // dI2/(2 s)
      v.dxi[p] = (p < 3 ? rs : 0.f) - v.xi * rs * v.ds[p];
    }
  } else {
    v.s = v.xi = 0.f;
#pragma unroll
    for (int p = 0; p < 6; ++p) v.ds[p] = v.dxi[p] = 0.f;
  }
  return v;
}

// Adds to lu[10] the gradient of sum_p ls[p] sigma_p(u) (sigma_p the six
// independent entries xx yy zz xy yz zx of the CDM stress); returns its xi0 part.
__device__ __forceinline__ float stress_vjp(const float* u, const MatF& m, const float ls[6], float lu[10]) {
  const Inv v = invariants(u);
  const float ag = u[9] * m.gamma_r;
  const float sh = 2.f * (m.mu0 + ag * m.xi0) - ag * v.xi;
  const float tr = ls[0] + ls[1] + ls[2];
  float le = 0.f;
#pragma unroll
  for (int p = 0; p < 6; ++p) le = fmaf(ls[p], u[p], le);
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const float diso = (p < 3 ? m.lam0 : 0.f) - ag * v.ds[p];
    lu[p] += tr * diso - le * ag * v.dxi[p] + sh * ls[p];
  }
  lu[9] += -tr * m.gamma_r * v.s + le * m.gamma_r * (2.f * m.xi0 - v.xi);
  return 2.f * le * ag;
}

// Adds to lu[0..5] the gradient of lr * r(u) (CDM damage rate); adds its xi0
// and C_d parts to *gx and *gc.
__device__ __forceinline__ void rate_vjp(const float* u, const MatF& m, float lr, float lu[10], float* gx,
                                         float* gc) {
  const Inv v = invariants(u);
  const float arg = v.I1 * v.s - m.xi0 * v.I2;
  if (!(arg > 0.f)) return;
  const float k = lr * m.cd * m.gamma_r;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const float d1 = p < 3 ? 1.f : 0.f, d2 = (p < 3 ? 2.f : 4.f) * u[p];
    lu[p] += k * (d1 * v.s + v.I1 * v.ds[p] - m.xi0 * d2);
  }
  *gx -= k * v.I2;
  *gc += lr * m.gamma_r * arg;
}

// Adds to lu[10] the gradient of sum_{d,p} lF[d][p] F^d_p(u) (flux of Eq.
// "nonlinear hyper pdes", lF [3][9] row-major); returns its xi0 part.
__device__ __forceinline__ float flux_vjp(const float* u, const MatF& m, const float* lF, float lu[10]) {
  // strain rows F^d_(ij) = -(v_i delta_jd + v_j delta_id) / 2
  lu[6] += -lF[0 * 9 + 0] - 0.5f * (lF[1 * 9 + 3] + lF[2 * 9 + 5]);
  lu[7] += -lF[1 * 9 + 1] - 0.5f * (lF[0 * 9 + 3] + lF[2 * 9 + 4]);
  lu[8] += -lF[2 * 9 + 2] - 0.5f * (lF[1 * 9 + 4] + lF[0 * 9 + 5]);
  // velocity rows F^d_(v_i) = -sigma_id / rho
  const float r = -m.rho_inv;
  const float ls[6] = {r * lF[0 * 9 + 6], r * lF[1 * 9 + 7], r * lF[2 * 9 + 8],
                       r * (lF[1 * 9 + 6] + lF[0 * 9 + 7]), r * (lF[2 * 9 + 7] + lF[1 * 9 + 8]),
                       r * (lF[0 * 9 + 8] + lF[2 * 9 + 6])};
  return stress_vjp(u, m, ls, lu);
}

// Adds to lu[10] the gradient of sum_p lf[p] (F(u) n)_p (the normal flux of the
// face kernel); returns its xi0 part.
__device__ __forceinline__ float normal_flux_vjp(const float* u, const MatF& m, const float n[3], const float lf[9],
                                                 float lu[10]) {
  lu[6] += -lf[0] * n[0] - 0.5f * (lf[3] * n[1] + lf[5] * n[2]);
  lu[7] += -lf[1] * n[1] - 0.5f * (lf[3] * n[0] + lf[4] * n[2]);
  lu[8] += -lf[2] * n[2] - 0.5f * (lf[4] * n[1] + lf[5] * n[0]);
  const float r = -m.rho_inv;
  const float ls[6] = {r * lf[6] * n[0], r * lf[7] * n[1], r * lf[8] * n[2], r * (lf[6] * n[1] + lf[7] * n[0]),
                       r * (lf[7] * n[2] + lf[8] * n[1]), r * (lf[6] * n[2] + lf[8] * n[0])};
  return stress_vjp(u, m, ls, lu);
}

// Transpose of the boundary flux of a free-surface (bc 1) or absorbing (bc 2) face
// (Appendix A; the closed form of the forward face kernel): adds to lu[10] the gradient
// of sum_p lf[p] F_p(u), which is linear in u, and to *dl and *dm its derivatives in the
// effective Lame parameters lambda and mu of the cell mean (through sigma_nn, c_p, c_s
// and k_p = c_p / (lambda + 2 mu)).
__device__ __forceinline__ void boundary_flux_vjp(int bc, const float* u, const float n[3], float lam, float mu,
                                                  float rho_inv, float cp, float cs, float kp, const float lf[9],
                                                  float lu[10], float* dl, float* dm) {
  const float En[3] = {u[0] * n[0] + u[3] * n[1] + u[5] * n[2], u[3] * n[0] + u[1] * n[1] + u[4] * n[2],
                       u[5] * n[0] + u[4] * n[1] + u[2] * n[2]};
  const float enn = En[0] * n[0] + En[1] * n[1] + En[2] * n[2];
  const float I1 = u[0] + u[1] + u[2];
  const float snn = lam * I1 + 2.f * mu * enn;
  const float vn = u[6] * n[0] + u[7] * n[1] + u[8] * n[2];
  float vt[3], et[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    vt[i] = u[6 + i] - vn * n[i];
    et[i] = En[i] - enn * n[i];
  }
  const float h = bc == 2 ? 0.5f : 1.f;
  // strain rows h (a n n^T + n b^T + b n^T)
  const float la = h * (lf[0] * n[0] * n[0] + lf[1] * n[1] * n[1] + lf[2] * n[2] * n[2] + lf[3] * n[0] * n[1] +
                        lf[4] * n[1] * n[2] + lf[5] * n[2] * n[0]);
  const float lb[3] = {h * (2.f * lf[0] * n[0] + lf[3] * n[1] + lf[5] * n[2]),
                       h * (2.f * lf[1] * n[1] + lf[3] * n[0] + lf[4] * n[2]),
                       h * (2.f * lf[2] * n[2] + lf[4] * n[1] + lf[5] * n[0])};
  float lsnn = 0.f, lvn = 0.f, lvt[3] = {0.f, 0.f, 0.f}, let[3] = {0.f, 0.f, 0.f};
  float dlam = 0.f, dmu = 0.f, dcp = 0.f, dcs = 0.f, dkp = 0.f;
  if (bc == 2) {
    // velocity rows pn n_i + (-2 mu et_i rho_inv + c_s vt_i) / 2, pn = (-sigma_nn rho_inv + c_p v.n) / 2
    const float lpn = lf[6] * n[0] + lf[7] * n[1] + lf[8] * n[2];
    lsnn += -0.5f * rho_inv * lpn;
    lvn += 0.5f * cp * lpn;
    dcp += 0.5f * vn * lpn;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      let[i] += -mu * rho_inv * lf[6 + i];
      lvt[i] += 0.5f * cs * lf[6 + i];
      dmu += -et[i] * rho_inv * lf[6 + i];
      dcs += 0.5f * vt[i] * lf[6 + i];
    }
  }
  // b_i = -vt_i / 2 + c_s et_i ; a = -v.n + k_p sigma_nn
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lvt[i] += -0.5f * lb[i];
    let[i] += cs * lb[i];
    dcs += lb[i] * et[i];
  }
  lvn += -la;
  lsnn += kp * la;
  dkp += la * snn;
  // et_i = En_i - enn n_i ; vt_i = v_i - vn n_i ; sigma_nn = lambda I1 + 2 mu enn ; vn = v.n ; enn = En.n
  float lEn[3], lenn = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lEn[i] = let[i];
    lenn -= let[i] * n[i];
    lvn -= lvt[i] * n[i];
  }
  const float lI1 = lam * lsnn;
  lenn += 2.f * mu * lsnn;
  dlam += lsnn * I1;
  dmu += 2.f * lsnn * enn;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lu[6 + i] += lvt[i] + lvn * n[i];
    lEn[i] += lenn * n[i];
  }
  // En_i = sum_j eps_ij n_j
  lu[0] += lEn[0] * n[0] + lI1;
  lu[1] += lEn[1] * n[1] + lI1;
  lu[2] += lEn[2] * n[2] + lI1;
  lu[3] += lEn[0] * n[1] + lEn[1] * n[0];
  lu[4] += lEn[1] * n[2] + lEn[2] * n[1];
  lu[5] += lEn[0] * n[2] + lEn[2] * n[0];
  // c_p = sqrt((lambda + 2 mu) rho_inv), c_s = sqrt(mu rho_inv), k_p = c_p / (lambda + 2 mu)
  const float m2 = lam + 2.f * mu;
  if (cp > 0.f && m2 > 0.f) {
    dlam += dcp * 0.5f * rho_inv / cp - dkp * 0.5f * kp / m2;
    dmu += dcp * rho_inv / cp - dkp * kp / m2;
  }
  if (cs > 0.f) dmu += dcs * 0.5f * rho_inv / cs;
  *dl += dlam;
  *dm += dmu;
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

// Block-wide sum of one float per thread into a shared double (atomic).
__device__ __forceinline__ void block_add(double* acc, float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(acc, static_cast<double>(v));
}

// Taylor coefficients c[z][o] = (tz_z dt)^o / o! and time weights gz_z dt of the
// step, once per CTA.
template <int N>
__device__ __forceinline__ void time_tables(const float* tb, const TableLayout& T, float dt, float* sC, float* sG) {
  constexpr int NT = N + 1;
  if (threadIdx.x < NT) {
    const int z = threadIdx.x;
    const float t = __ldg(tb + T.tz + z) * dt;
    float c = 1.f;
    for (int o = 0; o < NT; ++o) {
      if (o > 0) c *= t / static_cast<float>(o);
      sC[z * NT + o] = c;
    }
    sG[z] = __ldg(tb + T.gz + z) * dt;
  }
}

// Modes of Taylor order o held for field p: the wave fields of D^o have the
// modes of degree <= N - o, alpha has orders 0 and 1 on all modes.
template <int N>
__host__ __device__ constexpr int order_modes(int o, int p) {
  return p == 9 ? (o <= 1 ? n_modes(N) : 0) : n_modes(N - o);
}
// Offset of (o, l, p) in the (Q, D) layout of one element (Q stride q_stride(N)).
template <int N>
__device__ __forceinline__ int ld_index(int o, int l, int p) {
  if (o == 0) return l * 10 + p;
  if (p == 9) return q_stride(N) + d_alpha_offset(N) + l;
  return q_stride(N) + d_offset(N, o) + l * 9 + p;
}

// For two nodes x, x+1 of a basis table V[l][x] (row stride ldv) and field p: the mode
// sums t[o] = sum_l V[l][x] D^o_lp of every Taylor order o (D^0 = the state Q, row
// stride 10; D^o, o >= 1, row stride 9; alpha has orders 0 and 1 on all modes).  The
// loops run over compile-time mode counts and share each table load between orders.
template <int N>
__device__ __forceinline__ void mode_sums(const float* vx, int ldv, const float* Qs, const float* Ds, int p,
                                          float* t0, float* t1) {
  constexpr int NT = N + 1, L = n_modes(N);
#pragma unroll
  for (int o = 0; o < NT; ++o) t0[o] = t1[o] = 0.f;
  if (p == 9) {
#pragma unroll 4
    for (int l = 0; l < L; ++l) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(vx + l * ldv));
      const float c0 = Qs[l * 10 + 9], c1 = Ds[d_alpha_offset(N) + l];
      t0[0] = fmaf(v.x, c0, t0[0]);
      t1[0] = fmaf(v.y, c0, t1[0]);
      t0[1] = fmaf(v.x, c1, t0[1]);
      t1[1] = fmaf(v.y, c1, t1[1]);
    }
  } else {
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float2 v = __ldg(reinterpret_cast<const float2*>(vx + l * ldv));
#pragma unroll
      for (int o = 0; o < NT; ++o) {
        if (l < n_modes(N - o)) {
          const float c = o == 0 ? Qs[l * 10 + p] : Ds[d_offset(N, o) + l * 9 + p];
          t0[o] = fmaf(v.x, c, t0[o]);
          t1[o] = fmaf(v.y, c, t1[o]);
        }
      }
    }
  }
}

// The same for four nodes x..x+3 (ldv and x multiples of 4: one 16-byte table load per mode).
template <int N>
__device__ __forceinline__ void mode_sums4(const float* vx, int ldv, const float* Qs, const float* Ds, int p,
                                           float (*t)[N + 1]) {
  constexpr int NT = N + 1, L = n_modes(N);
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int o = 0; o < NT; ++o) t[n][o] = 0.f;
  if (p == 9) {
#pragma unroll 4
    for (int l = 0; l < L; ++l) {
      const float4 v4 = __ldg(reinterpret_cast<const float4*>(vx + l * ldv));
      const float v[4] = {v4.x, v4.y, v4.z, v4.w};
      const float c0 = Qs[l * 10 + 9], c1 = Ds[d_alpha_offset(N) + l];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        t[n][0] = fmaf(v[n], c0, t[n][0]);
        t[n][1] = fmaf(v[n], c1, t[n][1]);
      }
    }
  } else {
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const float4 v4 = __ldg(reinterpret_cast<const float4*>(vx + l * ldv));
      const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int o = 0; o < NT; ++o) {
        if (l < n_modes(N - o)) {
          const float c = o == 0 ? Qs[l * 10 + p] : Ds[d_offset(N, o) + l * 9 + p];
#pragma unroll
          for (int n = 0; n < 4; ++n) t[n][o] = fmaf(v[n], c, t[n][o]);
        }
      }
    }
  }
}

// Work items of node_values (per side): four nodes per item when the table's row
// stride is a multiple of 4, else two, times the ten fields.
template <int NX, int LDV>
__host__ __device__ constexpr int node_value_items() {
  return (LDV % 4 == 0 ? (NX + 3) / 4 : (NX + 1) / 2) * 10;
}

// For every node x of a basis table V[l][x] (row stride ldv, NX nodes) and field
// p: the value of the predictor's polynomial at the NT time nodes,
//     u[z][x][p] = sum_o c[z][o] sum_l V[l][x] D^o_lp,
// taking the sum over modes once per Taylor order.
template <int N, int NX, int LDV>
__device__ __forceinline__ void node_values(const float* V, const float* sQ, const float* sD, const float* sC,
                                            float* out, float* out0 = nullptr) {
  constexpr int NT = N + 1, NXH = (NX + 1) / 2;
  constexpr int ldv = LDV;
  if constexpr (LDV % 4 == 0) {
    // four nodes per item (the table's rows are padded with zeros to LDV >= NX)
    constexpr int NX4 = (NX + 3) / 4;
    for (int w = threadIdx.x; w < NX4 * 10; w += blockDim.x) {
      const int xq = w / 10, p = w - xq * 10, x = 4 * xq;
      float t[4][NT];
      mode_sums4<N>(V + x, ldv, sQ, sD, p, t);
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        if (x + n >= NX) continue;
        if (out0 != nullptr && p < 6) out0[(x + n) * 6 + p] = t[n][0];   // the strains at t_n
#pragma unroll
        for (int z = 0; z < NT; ++z) {
          float u = 0.f;
#pragma unroll
          for (int o = 0; o < NT; ++o) u = fmaf(sC[z * NT + o], t[n][o], u);
          out[(z * NX + x + n) * 10 + p] = u;
        }
      }
    }
  } else {
  // two nodes per item: the table's rows are padded to an even length with zeros
  for (int w = threadIdx.x; w < NXH * 10; w += blockDim.x) {
    const int xh = w / 10, p = w - xh * 10, x = 2 * xh;
    const float* vx = V + x;
    float t0[NT], t1[NT];
    mode_sums<N>(vx, ldv, sQ, sD, p, t0, t1);
    const bool two = x + 1 < NX;
    if (out0 != nullptr && p < 6) {                           // the strains at t_n
      out0[x * 6 + p] = t0[0];
      if (two) out0[(x + 1) * 6 + p] = t1[0];
    }
#pragma unroll
    for (int z = 0; z < NT; ++z) {
      float u0 = 0.f, u1 = 0.f;
#pragma unroll
      for (int o = 0; o < NT; ++o) {
        u0 = fmaf(sC[z * NT + o], t0[o], u0);
        u1 = fmaf(sC[z * NT + o], t1[o], u1);
      }
      out[(z * NX + x) * 10 + p] = u0;
      if (two) out[(z * NX + x + 1) * 10 + p] = u1;
    }
  }
  }
}

// node_values for the two sides of a face in one pass (items over both sides): side s
// takes its table V[s] and its element's state Q + s QS and predictor output D + s DS.
template <int N, int NX, int LDV>
__device__ __forceinline__ void node_values_2side(const float* V0, const float* V1, const float* sQ,
                                                  const float* sD, const float* sC, float* out) {
  constexpr int NT = N + 1, NXH = (NX + 1) / 2, QS = q_stride(N), DS = d_stride(N);
  constexpr int ldv = LDV;
  if constexpr (LDV % 4 == 0) {
    constexpr int NX4 = (NX + 3) / 4;
    for (int w = threadIdx.x; w < 2 * NX4 * 10; w += blockDim.x) {
      const int sd = w / (NX4 * 10), r = w - sd * NX4 * 10;
      const int xq = r / 10, p = r - xq * 10, x = 4 * xq;
      float t[4][NT];
      mode_sums4<N>((sd ? V1 : V0) + x, ldv, sQ + sd * QS, sD + sd * DS, p, t);
      float* os = out + sd * NT * NX * 10;
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        if (x + n >= NX) continue;
#pragma unroll
        for (int z = 0; z < NT; ++z) {
          float u = 0.f;
#pragma unroll
          for (int o = 0; o < NT; ++o) u = fmaf(sC[z * NT + o], t[n][o], u);
          os[(z * NX + x + n) * 10 + p] = u;
        }
      }
    }
  } else {
  for (int w = threadIdx.x; w < 2 * NXH * 10; w += blockDim.x) {
    const int sd = w / (NXH * 10), r = w - sd * NXH * 10;
    const int xh = r / 10, p = r - xh * 10, x = 2 * xh;
    const float* vx = (sd ? V1 : V0) + x;
    const float* Qs = sQ + sd * QS;
    const float* Ds = sD + sd * DS;
    float t0[NT], t1[NT];
    mode_sums<N>(vx, ldv, Qs, Ds, p, t0, t1);
    const bool two = x + 1 < NX;
    float* os = out + sd * NT * NX * 10;
#pragma unroll
    for (int z = 0; z < NT; ++z) {
      float u0 = 0.f, u1 = 0.f;
#pragma unroll
      for (int o = 0; o < NT; ++o) {
        u0 = fmaf(sC[z * NT + o], t0[o], u0);
        u1 = fmaf(sC[z * NT + o], t1[o], u1);
      }
      os[(z * NX + x) * 10 + p] = u0;
      if (two) os[(z * NX + x + 1) * 10 + p] = u1;
    }
  }
  }
}

// ---------------------------------------------------------------------------
// Faces
// ---------------------------------------------------------------------------
template <int N>
struct FaceSmem {
  using A = ADim<N>;
  static constexpr int oLam = 0;                              // [2][QS] lam^{k+1} of both sides
  static constexpr int oQ = oLam + 2 * A::QS;                 // [2][QS]
  static constexpr int oD = oQ + 2 * A::QS;                   // [2][DS]
  static constexpr int oTr = oD + 2 * A::DS;                  // [2][NT][NF][10] traces
  static constexpr int oLff = round4(oTr + 2 * A::NT * A::NF * 10);   // [NF][9]
  static constexpr int oLu = round4(oLff + A::NF * 9);        // [2][NT][NF][10] lam of the traces,
                                                              //   then folded into Taylor orders
  static constexpr int total = oLu + 2 * A::NT * A::NF * 10;
};

template <int N>
__global__ void __launch_bounds__(128, 8) k_adj_face(AdjArgs a) {
  using A = ADim<N>;
  using S = FaceSmem<N>;
  constexpr int L = A::L, NF = A::NF, NT = A::NT;
  extern __shared__ __align__(16) float smem[];
  __shared__ double sRed[6];
  __shared__ float sC[NT * NT], sG[NT], sIB[NF];
  const TableLayout T = table_layout(N);
  const float* tb = a.tables;
  time_tables<N>(tb, T, a.dt, sC, sG);
  // 1 / beta_i of the face rule: beta_i phi_0 is column 0 of any local face's weighted table
  for (int i = threadIdx.x; i < NF; i += blockDim.x) sIB[i] = 2.449489742783178f / __ldg(tb + T.Vfw + i * A::LP);
  for (int64_t f = blockIdx.x; f < a.F; f += gridDim.x) {
    const int4 fc = a.faces[f];
    // a boundary face is (element, local face, -1, tag): its side 1 is a stand-in that
    // receives nothing
    const bool bnd = fc.z < 0;
    const int bc = bnd ? fc.w : 0;
    const int64_t e0 = fc.x, e1 = bnd ? fc.x : fc.z;
    const int lf0 = fc.y, lf1 = bnd ? fc.y : fc.w;
    __syncthreads();
    // one batch of 16-byte asynchronous copies: lam, Q and D of both sides
    for (int w = threadIdx.x; w < A::QS / 2; w += blockDim.x) {
      const int sd = w / (A::QS / 4), c = 4 * (w - sd * (A::QS / 4));
      const int64_t es = sd ? e1 : e0;
      tc::cp_async16(smem + S::oLam + sd * A::QS + c, a.lam_in + es * A::QS + c);
      tc::cp_async16(smem + S::oQ + sd * A::QS + c, a.q + es * A::QS + c);
    }
    for (int w = threadIdx.x; w < A::DS / 2; w += blockDim.x) {
      const int sd = w / (A::DS / 4), c = 4 * (w - sd * (A::DS / 4));
      tc::cp_async16(smem + S::oD + sd * A::DS + c, a.d + (sd ? e1 : e0) * A::DS + c);
    }
    tc::cp_async_wait_all();
    if (threadIdx.x < 6) sRed[threadIdx.x] = 0.0;
    __syncthreads();
    // traces of both sides at the space-time face nodes
    // the traces and lam of the face flux (independent of each other) in one phase
    node_values_2side<N, NF, A::NFP>(tb + T.VfT + lf0 * L * A::NFP, tb + T.VfT + lf1 * L * A::NFP, smem + S::oQ,
                                     smem + S::oD, sC, smem + S::oTr);
    // lam of the time-integrated face flux:
    //   lff[i][p] = -(a0 sum_k Vfw[f0][i][k] lam0[k][p] - a1 sum_k Vfw[f1][i][k] lam1[k][p])
    const float a0 = a.geom[e0].face[lf0][3], a1 = bnd ? 0.f : a.geom[e1].face[lf1][3];
    // the items continue the traces' round-robin over the threads, so that the threads
    // without a trace item take the first ones
    constexpr int NVI = 2 * node_value_items<NF, A::NFP>();
    for (int w = (threadIdx.x + blockDim.x - NVI % blockDim.x) % blockDim.x; w < NF * 9; w += blockDim.x) {
      const int i = w / 9, p = w - i * 9;
      const float4* v0 = reinterpret_cast<const float4*>(tb + T.Vfw + (lf0 * NF + i) * A::LP);
      const float4* v1 = reinterpret_cast<const float4*>(tb + T.Vfw + (lf1 * NF + i) * A::LP);
      const float* l0 = smem + S::oLam + p;
      const float* l1 = smem + S::oLam + A::QS + p;
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int kq = 0; kq < A::LP / 4; ++kq) {
        const float4 x = __ldg(v0 + kq), y = __ldg(v1 + kq);
        const int k = 4 * kq;
        // the table's rows are zero beyond L; lam is read only at modes below L
        s0 = fmaf(x.x, l0[k * 10], s0);
        s1 = fmaf(y.x, l1[k * 10], s1);
        if (k + 1 < L) { s0 = fmaf(x.y, l0[(k + 1) * 10], s0); s1 = fmaf(y.y, l1[(k + 1) * 10], s1); }
        if (k + 2 < L) { s0 = fmaf(x.z, l0[(k + 2) * 10], s0); s1 = fmaf(y.z, l1[(k + 2) * 10], s1); }
        if (k + 3 < L) { s0 = fmaf(x.w, l0[(k + 3) * 10], s0); s1 = fmaf(y.w, l1[(k + 3) * 10], s1); }
      }
      smem[S::oLff + w] = -(a0 * s0 - a1 * s1);
    }
    __syncthreads();
    // the Rusanov flux (or the boundary flux) transposed at each space-time node, one side per item
    const float n[3] = {a.geom[e0].face[lf0][0], a.geom[e0].face[lf0][1], a.geom[e0].face[lf0][2]};
    const float cp0 = a.cp[e0], cp1 = a.cp[e1];
    const float C = fmaxf(cp0, cp1);
    // boundary faces: effective Lame parameters of the own cell mean and the speeds of the forward flux
    float blam = 0.f, bmu = 0.f, bcp = 0.f, bcs = 0.f, bkp = 0.f;
    const MatF mb = a.mat[e0];
    if (bnd) {
      const float r6 = 2.449489742783178f;
      float ub[10];
#pragma unroll
      for (int p = 0; p < 10; ++p) ub[p] = smem[S::oQ + p] * r6;
      const Inv v = invariants(ub);
      blam = mb.lam0 - ub[9] * mb.gamma_r * v.xi * (1.f / 3.f);
      bmu = mb.mu0 + ub[9] * mb.xi0 * mb.gamma_r - 0.5f * ub[9] * mb.gamma_r * v.xi;
      bcp = sqrtf(fmaxf(blam + 2.f * bmu, 0.f) * mb.rho_inv);
      bcs = sqrtf(fmaxf(bmu, 0.f) * mb.rho_inv);
      bkp = blam + 2.f * bmu > 0.f ? bcp / (blam + 2.f * bmu) : 0.f;
    }
    float pC = 0.f, px0 = 0.f, px1 = 0.f, pl = 0.f, pm = 0.f;
    for (int w = threadIdx.x; w < 2 * NT * NF; w += blockDim.x) {
      const int sd = w / (NT * NF), r = w - sd * NT * NF;
      const int z = r / NF, i = r - z * NF;
      const float g = sG[z];
      const float* u = smem + S::oTr + w * 10;
      float lfs[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) lfs[p] = g * smem[S::oLff + i * 9 + p];
      float lu[10];
#pragma unroll
      for (int p = 0; p < 10; ++p) lu[p] = 0.f;
      float* o = smem + S::oLu + w * 10;
      if (bnd) {
        if (sd == 0) boundary_flux_vjp(bc, u, n, blam, bmu, mb.rho_inv, bcp, bcs, bkp, lfs, lu, &pl, &pm);
#pragma unroll
        for (int p = 0; p < 9; ++p) o[p] = lu[p];
        o[9] = 0.f;
        continue;
      }
      const MatF m = a.mat[sd ? e1 : e0];
      const float gx = 0.5f * normal_flux_vjp(u, m, n, lfs, lu);
      const float cs = sd ? -0.5f * C : 0.5f * C;
#pragma unroll
      for (int p = 0; p < 9; ++p) o[p] = 0.5f * lu[p] + cs * lfs[p];
      o[9] = 0.5f * lu[9];
      if (sd == 0) {
        px0 += gx;
        const float* up = smem + S::oTr + (NT * NF + r) * 10;
#pragma unroll
        for (int p = 0; p < 9; ++p) pC = fmaf(0.5f * lfs[p], u[p] - up[p], pC);
      } else {
        px1 += gx;
      }
    }
    block_add(&sRed[3], pl);
    block_add(&sRed[4], pm);
    block_add(&sRed[0], pC);
    block_add(&sRed[1], px0);
    block_add(&sRed[2], px1);
    __syncthreads();
    // fold the time nodes into Taylor orders in place, divided by the face weight of the
    // node (the projection below runs over beta_i phi_l(x_i)):
    //   Lo[o][i][p] = sum_z c[z][o] Lu[z][i][p] / beta_i,  beta_i = Vfw[.][i][0] / phi_0
    for (int w = threadIdx.x; w < 2 * NF * 10; w += blockDim.x) {
      const int sd = w / (NF * 10), r = w - sd * NF * 10;
      const float ib = sIB[r / 10];
      float* base = smem + S::oLu + sd * NT * NF * 10 + r;
      float lz[NT];
#pragma unroll
      for (int z = 0; z < NT; ++z) lz[z] = base[z * NF * 10];
#pragma unroll
      for (int o = 0; o < NT; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int z = 0; z < NT; ++z) acc = fmaf(sC[z * NT + o], lz[z], acc);
        base[o * NF * 10] = acc * ib;
      }
    }
    __syncthreads();
    // lam of D^o_lp of each side = sum_i beta_i phi_l(x_i) Lo[o][i][p]; one item per four
    // modes and pair of fields (16-byte loads of the node-major weighted table)
    constexpr int LQ = A::LP / 4, PITEMS = 2 * LQ * 5 * 2;   // (side, 4 modes, pair of fields, half of the nodes)
    for (int base = 0; base < PITEMS; base += blockDim.x) {   // warp-uniform trip count (shuffles below)
      const int w = base + threadIdx.x;
      const bool live = w < PITEMS;
      const int item = live ? w >> 1 : 0, ic = w & 1;
      const int sd = item / (LQ * 5), r = item - sd * LQ * 5, lq = r / 5, p0 = 2 * (r - lq * 5);
      const float4* V = reinterpret_cast<const float4*>(tb + T.Vfw + (sd ? lf1 : lf0) * NF * A::LP) + lq;
      const float* Lo = smem + S::oLu + sd * NT * NF * 10 + p0;
      float acc[4][2][NT];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int o = 0; o < NT; ++o) acc[j][0][o] = acc[j][1][o] = 0.f;
#pragma unroll 2
      for (int i = live ? ic : NF; i < NF; i += 2) {
        const float4 v4 = __ldg(V + i * LQ);
        const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int o = 0; o < NT; ++o) {
          const float2 lo = *reinterpret_cast<const float2*>(Lo + (o * NF + i) * 10);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[j][0][o] = fmaf(v[j], lo.x, acc[j][0][o]);
            acc[j][1][o] = fmaf(v[j], lo.y, acc[j][1][o]);
          }
        }
      }
      // the two node halves of an item sit on adjacent lanes: their sums, with lane ic left
      // holding modes 4 lq + 2 ic and 4 lq + 2 ic + 1 (each sends the pair it does not keep)
      float s2[2][2][NT];
#pragma unroll
      for (int jj = 0; jj < 2; ++jj)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int o = 0; o < NT; ++o) {
            const float keep = ic ? acc[2 + jj][h][o] : acc[jj][h][o];
            const float send = ic ? acc[jj][h][o] : acc[2 + jj][h][o];
            s2[jj][h][o] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
          }
      if (!live) continue;
      float* out = a.rec + (f * 2 + sd) * A::RS;
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int l = 4 * lq + 2 * ic + jj;
        if (l >= L) continue;
#pragma unroll
        for (int o = 0; o < NT; ++o) {
          if (l < order_modes<N>(o, p0)) out[ld_index<N>(o, l, p0)] = s2[jj][0][o];
          if (l < order_modes<N>(o, p0 + 1)) out[ld_index<N>(o, l, p0 + 1)] = s2[jj][1][o];
        }
      }
    }
    if (threadIdx.x < 2) {
      const int sd = threadIdx.x;
      // C = max(cp0, cp1): its derivative goes to the larger speed, in halves at a tie
      const float share = cp0 > cp1 ? (sd == 0 ? 1.f : 0.f) : (cp0 < cp1 ? (sd == 1 ? 1.f : 0.f) : 0.5f);
      float* tail = a.rec + (f * 2 + sd) * A::RS + A::LDS;
      // lam of the side's P speed, the xi0 part of its flux, and (boundary faces) the flux's
      // derivatives in the own cell's lambda_eff and mu_eff
      tail[0] = bnd ? 0.f : share * static_cast<float>(sRed[0]);
      tail[1] = bnd ? 0.f : static_cast<float>(sRed[1 + sd]);
      tail[2] = bnd && sd == 0 ? static_cast<float>(sRed[3]) : 0.f;
      tail[3] = bnd && sd == 0 ? static_cast<float>(sRed[4]) : 0.f;
    }
  }
}

// ---------------------------------------------------------------------------
// Elements
// ---------------------------------------------------------------------------
template <int N>
struct ElemSmem {
  using A = ADim<N>;
  static constexpr int oLam = 0;                          // [L][10] lam^{k+1}
  static constexpr int oQ = round4(oLam + A::L * 10);     // [QS]
  static constexpr int oD = oQ + A::QS;                   // [DS]
  static constexpr int oU = oD + A::DS;                   // [NT][NQ][10] nodal values, then their lam
  static constexpr int oLu = oU;                          //   (each node's lam replaces its value)
  static constexpr int oX = round4(oU + A::NT * A::NQ * 10);   // [NQ][28]: w_q dphi_k/dx_d lam_kp (27), w_q phi_k lam_k9
  static constexpr int oLD = oX + A::NQ * 28;             // [QS + DS] lam of D^0..D^N
  // [3][9][LP] H of the CK transpose, mode fastest: in the X region, after the forward CK
  // products (both live only from the projection on)
  static constexpr int oH = oX + round4(27 * A::GXI);
  static_assert(round4(27 * A::GXI) + 27 * A::LP <= A::NQ * 28, "CK products and H inside the X region");
  static constexpr int oR = round4(oLD + A::LDS);         // [4][RS] the element's four face records
  static constexpr int total = oR + 4 * A::RS;
};

template <int N>
__global__ void __launch_bounds__(128, 7) k_adj_elem(AdjArgs a) {
  using A = ADim<N>;
  using S = ElemSmem<N>;
  constexpr int L = A::L, NQ = A::NQ, NT = A::NT;
  extern __shared__ __align__(16) float smem[];
  // xi0, C_d, lam of cp, (unused), boundary d/dlam, d/dmu, CK d/d(lam/rho), CK d/d(mu/rho)
  __shared__ double sRed[8];
  __shared__ float sGeo[16];          // Theta^{-1} [e][d]; lambda_eff, mu_eff of the cell mean at [9], [10]
  __shared__ float sC[NT * NT], sG[NT], sIW[NQ];
  const TableLayout T = table_layout(N);
  const float* tb = a.tables;
  time_tables<N>(tb, T, a.dt, sC, sG);
  // 1 / w_q of the volume rule: w_q phi_0 is column 0 of the weighted table
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) sIW[q] = 2.449489742783178f / __ldg(tb + T.Vw + q * A::LP);
  float* sLD = smem + S::oLD;
  for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
    __syncthreads();
    // two groups of 16-byte asynchronous copies: lam, Q and D, then the four face records
    // (first needed by the projection, so that their gather overlaps the nodal phases)
    {
      const int4 ef4 = reinterpret_cast<const int4*>(a.elem_face)[e];
      for (int w = threadIdx.x; w < A::QS / 4; w += blockDim.x) {
        tc::cp_async16(smem + S::oLam + 4 * w, a.lam_in + e * A::QS + 4 * w);
        tc::cp_async16(smem + S::oQ + 4 * w, a.q + e * A::QS + 4 * w);
      }
      for (int w = threadIdx.x; w < A::DS / 4; w += blockDim.x)
        tc::cp_async16(smem + S::oD + 4 * w, a.d + e * A::DS + 4 * w);
      tc::cp_async_commit();
      for (int w = threadIdx.x; w < A::RS; w += blockDim.x) {
        const int fl = w / (A::RS / 4), c = 4 * (w - fl * (A::RS / 4));
        const int ef = fl == 0 ? ef4.x : (fl == 1 ? ef4.y : (fl == 2 ? ef4.z : ef4.w));
        tc::cp_async16(smem + S::oR + fl * A::RS + c, a.rec + static_cast<int64_t>(ef) * A::RS + c);
      }
    }
    tc::cp_async_commit();
    // (sLD needs no zeroing: the projection assigns every entry that is read later)
    tc::cp_async_wait<1>();                  // lam, Q, D have landed; the records may still be in flight
    const MatF m = a.mat[e];
    if (threadIdx.x < 9) sGeo[threadIdx.x] = a.geom[e].tinv[threadIdx.x];
    if (threadIdx.x < 8) sRed[threadIdx.x] = 0.0;
    __syncthreads();
    // the nodal values and X (independent of each other) in one phase
    node_values<N, NQ, A::NQP>(tb + T.VvT, smem + S::oQ, smem + S::oD, sC, smem + S::oU);
    // per volume node q: X[q][d][p] = sum_k w_q dphi_k/dx_d(x_q) lam[k][p], X[q][27] = sum_k w_q phi_k lam[k][9];
    // one item per node and pair of fields (8, 9 pairs the last wave field with alpha); the
    // items continue the nodal values' round-robin over the threads
    constexpr int NVI = node_value_items<NQ, A::NQP>();
    for (int w = (threadIdx.x + blockDim.x - NVI % blockDim.x) % blockDim.x; w < NQ * 5; w += blockDim.x) {
      const int q = w / 5, pp = w - q * 5, p0 = 2 * pp;
      float g0[3] = {0.f, 0.f, 0.f}, g1[3] = {0.f, 0.f, 0.f};
      const float4* gA = reinterpret_cast<const float4*>(tb + T.Gw + q * A::LP);
      const float4* gB = reinterpret_cast<const float4*>(tb + T.Gw + (NQ + q) * A::LP);
      const float4* gC = reinterpret_cast<const float4*>(tb + T.Gw + (2 * NQ + q) * A::LP);
      const float4* vW = reinterpret_cast<const float4*>(tb + T.Vw + q * A::LP);
#pragma unroll
      for (int kq = 0; kq < A::LP / 4; ++kq) {
        // lam at modes 4 kq .. 4 kq + 3 of fields p0, p0 + 1 (zero beyond L, where the tables are zero too)
        float xv[4], yv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = 4 * kq + j;
          const float2 lk = k < L ? *reinterpret_cast<const float2*>(smem + S::oLam + k * 10 + p0) : make_float2(0.f, 0.f);
          xv[j] = lk.x;
          yv[j] = lk.y;
        }
        const float4 x = make_float4(xv[0], xv[1], xv[2], xv[3]), y = make_float4(yv[0], yv[1], yv[2], yv[3]);
        const float4 ga = __ldg(gA + kq), gb = __ldg(gB + kq), gc = __ldg(gC + kq);
        g0[0] = dot4(ga, x, g0[0]);
        g0[1] = dot4(gb, x, g0[1]);
        g0[2] = dot4(gc, x, g0[2]);
        if (pp < 4) {
          g1[0] = dot4(ga, y, g1[0]);
          g1[1] = dot4(gb, y, g1[1]);
          g1[2] = dot4(gc, y, g1[2]);
        } else {
          g1[0] = dot4(__ldg(vW + kq), y, g1[0]);
        }
      }
      float* xq = smem + S::oX + q * 28;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        xq[d * 9 + p0] = g0[0] * sGeo[0 * 3 + d] + g0[1] * sGeo[1 * 3 + d] + g0[2] * sGeo[2 * 3 + d];
      if (pp < 4) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          xq[d * 9 + p0 + 1] = g1[0] * sGeo[0 * 3 + d] + g1[1] * sGeo[1 * 3 + d] + g1[2] * sGeo[2 * 3 + d];
      } else {
        xq[27] = g1[0];
      }
    }
    __syncthreads();
    // the volume flux and the damage-rate source transposed at each space-time volume node
    float px = 0.f, pc = 0.f;
    for (int w = threadIdx.x; w < NT * NQ; w += blockDim.x) {
      const int z = w / NQ, q = w - z * NQ;
      const float g = sG[z];
      float u[10];
#pragma unroll
      for (int p = 0; p < 10; p += 2) {
        const float2 v2 = *reinterpret_cast<const float2*>(smem + S::oU + w * 10 + p);
        u[p] = v2.x;
        u[p + 1] = v2.y;
      }
      float lF[28];
#pragma unroll
      for (int c = 0; c < 28; c += 4) {
        const float4 v4 = *reinterpret_cast<const float4*>(smem + S::oX + q * 28 + c);
        lF[c] = g * v4.x; lF[c + 1] = g * v4.y; lF[c + 2] = g * v4.z; lF[c + 3] = g * v4.w;
      }
      float lu[10];
#pragma unroll
      for (int p = 0; p < 10; ++p) lu[p] = 0.f;
      px += flux_vjp(u, m, lF, lu);
      rate_vjp(u, m, lF[27], lu, &px, &pc);
      // divided by the volume weight of the node: the projection runs over w_q phi_l(x_q)
      const float iw = sIW[q];
      float* o = smem + S::oLu + w * 10;
#pragma unroll
      for (int p = 0; p < 10; p += 2) *reinterpret_cast<float2*>(o + p) = make_float2(lu[p] * iw, lu[p + 1] * iw);
    }
    tc::cp_async_wait<0>();                  // the face records
    __syncthreads();
    // lam of D^o_lp = sum_z c[z][o] sum_q w_q phi_l(x_q) Lu[z][q][p] (Lu divided by w_q above),
    // plus the four face records; one item per four modes and pair of fields (16-byte loads
    // of the node-major weighted table)
    constexpr int LQ = A::LP / 4, PITEMS = LQ * 5 * 4;   // (4 modes, pair of fields, quarter of the nodes)
    for (int base = 0; base < PITEMS; base += blockDim.x) {   // warp-uniform trip count (shuffles below)
      const int w = base + threadIdx.x;
      const bool live = w < PITEMS;
      const int item = live ? w >> 2 : 0, qc = w & 3;
      const int lq = item / 5, p0 = 2 * (item - lq * 5);
      const float4* V = reinterpret_cast<const float4*>(tb + T.Vw) + lq;
      const float* Lu = smem + S::oLu + p0;
      float acc[4][2][NT];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int z = 0; z < NT; ++z) acc[j][0][z] = acc[j][1][z] = 0.f;
#pragma unroll 2
      for (int q = live ? qc : NQ; q < NQ; q += 4) {
        const float4 v4 = __ldg(V + q * LQ);
        const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int z = 0; z < NT; ++z) {
          const float2 lz = *reinterpret_cast<const float2*>(Lu + (z * NQ + q) * 10);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[j][0][z] = fmaf(v[j], lz.x, acc[j][0][z]);
            acc[j][1][z] = fmaf(v[j], lz.y, acc[j][1][z]);
          }
        }
      }
      // the four node quarters of an item sit on consecutive lanes: their sums, with lane
      // qc left holding mode 4 lq + qc (each exchange sends the half a lane does not keep)
      const bool hi2 = (qc & 2) != 0, hi1 = (qc & 1) != 0;
      float t2[2][2][NT];
#pragma unroll
      for (int jj = 0; jj < 2; ++jj)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int z = 0; z < NT; ++z) {
            const float keep = hi2 ? acc[2 + jj][h][z] : acc[jj][h][z];
            const float send = hi2 ? acc[jj][h][z] : acc[2 + jj][h][z];
            t2[jj][h][z] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
          }
      float t1[2][NT];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int z = 0; z < NT; ++z) {
          const float keep = hi1 ? t2[1][h][z] : t2[0][h][z];
          const float send = hi1 ? t2[0][h][z] : t2[1][h][z];
          t1[h][z] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
        }
      const int l = 4 * lq + qc;
      if (!live || l >= L) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = p0 + h;
#pragma unroll
        for (int o = 0; o < NT; ++o) {
          if (l >= order_modes<N>(o, p)) continue;
          float s = 0.f;
#pragma unroll
          for (int z = 0; z < NT; ++z) s = fmaf(sC[z * NT + o], t1[h][z], s);
          const int idx = ld_index<N>(o, l, p);
#pragma unroll
          for (int fl = 0; fl < 4; ++fl) s += smem[S::oR + fl * A::RS + idx];
          sLD[idx] = s;
        }
      }
    }
    // the forward CK products every order of the transposed recursion needs (they do not
    // depend on lam), computed here with many items instead of inside the order loop:
    // GX[i][k][q][d] = sum_e Theta^{-1}_ed sum_l Kt^e_kl D^{i-1}_lq, k < L_{N-i}, q < 9, in the
    // X region (free since the flux phase)
    {
      float* sGX = smem + S::oX;
      for (int w = threadIdx.x; w < A::GXI * 9; w += blockDim.x) {
#pragma unroll
        for (int i = 1; i <= N; ++i) {
          const int r0 = 9 * A::gx_row(i), r1 = 9 * A::gx_row(i + 1);
          if (w < r0 || w >= r1) continue;
          const int k = (w - r0) / 9, q = (w - r0) - 9 * k;
          const float* Dprev = i == 1 ? smem + S::oQ : smem + S::oD + d_offset(N, i - 1);
          const int sp = i == 1 ? 10 : 9;
          float gk0 = 0.f, gk1 = 0.f, gk2 = 0.f;
          const float* kt = tb + T.KtA + k;
#pragma unroll
          for (int l = 0; l < n_modes(N - i + 1); ++l) {
            const float dv = Dprev[l * sp + q];
            gk0 = fmaf(__ldg(kt + (0 * L + l) * A::LP), dv, gk0);
            gk1 = fmaf(__ldg(kt + (1 * L + l) * A::LP), dv, gk1);
            gk2 = fmaf(__ldg(kt + (2 * L + l) * A::LP), dv, gk2);
          }
          float* g = sGX + w * 3;
#pragma unroll
          for (int d = 0; d < 3; ++d) g[d] = sGeo[0 * 3 + d] * gk0 + sGeo[1 * 3 + d] * gk1 + sGeo[2 * 3 + d] * gk2;
        }
      }
    }
    if (threadIdx.x < 4) {
      const float* tail = smem + S::oR + threadIdx.x * A::RS + A::LDS;
      atomicAdd(&sRed[2], static_cast<double>(tail[0]));   // lam of cp (scaled below)
      atomicAdd(&sRed[0], static_cast<double>(tail[1]));   // xi0 part of the face fluxes
      atomicAdd(&sRed[4], static_cast<double>(tail[2]));   // boundary fluxes: d/dlambda_eff
      atomicAdd(&sRed[5], static_cast<double>(tail[3]));   //                  d/dmu_eff
    }
    block_add(&sRed[0], px);
    block_add(&sRed[1], pc);
    // effective Lame parameters of the cell mean (the forward predictor's rule), on the last
    // thread (no more items of the forward CK products than any other), shared after the barrier
    if (threadIdx.x == blockDim.x - 1) {
      const float r6 = 2.449489742783178f;
      float ub[10];
#pragma unroll
      for (int p = 0; p < 10; ++p) ub[p] = smem[S::oQ + p] * r6;
      const Inv v = invariants(ub);
      sGeo[9] = m.lam0 - ub[9] * m.gamma_r * v.xi * (1.f / 3.f);
      sGeo[10] = m.mu0 + ub[9] * m.xi0 * m.gamma_r - 0.5f * ub[9] * m.gamma_r * v.xi;
    }
    __syncthreads();                         // the projection's lam of D is complete
    const float lam_eff = sGeo[9], mu_eff = sGeo[10];
    // Cauchy-Kovalevskaya recursion transposed, order N down to 1 (the forward products in
    // GX; the lambda/rho and mu/rho parts summed per thread over all orders, reduced once)
    const float lr = lam_eff * m.rho_inv, mr = mu_eff * m.rho_inv;
    float plr = 0.f, pmr = 0.f;
    // the damage-rate source of D^1 from the state at t_n runs alongside the first order: it
    // reads only lam of D^1 of alpha (which the recursion does not change) and the strains at
    // t_n, and leaves its result in sDS, added to lam of the strains at the end
    //   lam_r(q) = sum_k w_q phi_k(x_q) lam D^1_k9;  lam Q_lp += sum_q phi_l(x_q) (d r / d eps_p)(q) lam_r(q)
    float* sLu0 = smem + S::oLu;               // [6][U0S] (reuses the nodal lam), node fastest
    float* sDS = smem + S::oLu + 6 * A::U0S;   // [L][6]
    float pxr = 0.f, pcr = 0.f;
#pragma unroll
    for (int i = N; i >= 1; --i) {
      const int Lout = n_modes(N - i), Lin = n_modes(N - i + 1);
      const float* lDi = sLD + A::QS + d_offset(N, i);       // [Lout][9]
      if (i == N) {
        // from the first warp without an H item below
        constexpr int Q0 = (9 * n_modes(0) + 31) / 32 * 32;
        for (int q = (threadIdx.x + blockDim.x - Q0 % blockDim.x) % blockDim.x; q < NQ; q += blockDim.x) {
          // the strains at t_n at node q, and lam of the damage rate there,
          //   w_q sum_k phi_k(x_q) lam D^1_k9
          float u[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          float lsum = 0.f;
#pragma unroll 4
          for (int l = 0; l < L; ++l) {
            const float v = __ldg(tb + T.VvT + l * A::NQP + q);
#pragma unroll
            for (int p = 0; p < 6; ++p) u[p] = fmaf(v, smem[S::oQ + l * 10 + p], u[p]);
            lsum = fmaf(v, sLD[A::QS + A::AOFF + l], lsum);
          }
          const float lrq = lsum / sIW[q];
          float lu[10];
#pragma unroll
          for (int p = 0; p < 10; ++p) lu[p] = 0.f;
          rate_vjp(u, m, lrq, lu, &pxr, &pcr);
#pragma unroll
          for (int p = 0; p < 6; ++p) sLu0[p * A::U0S + q] = lu[p];
        }
      }
      float* lDprev = i == 1 ? sLD : sLD + A::QS + d_offset(N, i - 1);
      const int lsp = i == 1 ? 10 : 9;
      const float* gxi = smem + S::oX + 27 * A::gx_row(i);
      for (int w = threadIdx.x; w < Lout * 9; w += blockDim.x) {
        const int k = w / 9, q = w - k * 9;
        float lv[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) lv[p] = lDi[k * 9 + p];
        // column q of Psi_d = B^d^T lam
        float ps[3];
        if (q < 3) {
#pragma unroll
          for (int d = 0; d < 3; ++d) ps[d] = -lr * lv[6 + d] - (q == d ? 2.f * mr * lv[6 + d] : 0.f);
        } else if (q == 3) {
          ps[0] = -2.f * mr * lv[7]; ps[1] = -2.f * mr * lv[6]; ps[2] = 0.f;
        } else if (q == 4) {
          ps[0] = 0.f; ps[1] = -2.f * mr * lv[8]; ps[2] = -2.f * mr * lv[7];
        } else if (q == 5) {
          ps[0] = -2.f * mr * lv[8]; ps[1] = 0.f; ps[2] = -2.f * mr * lv[6];
        } else if (q == 6) {
          ps[0] = -lv[0]; ps[1] = -0.5f * lv[3]; ps[2] = -0.5f * lv[5];
        } else if (q == 7) {
          ps[0] = -0.5f * lv[3]; ps[1] = -lv[1]; ps[2] = -0.5f * lv[4];
        } else {
          ps[0] = -0.5f * lv[5]; ps[1] = -0.5f * lv[4]; ps[2] = -lv[2];
        }
#pragma unroll
        for (int ee = 0; ee < 3; ++ee)
          smem[S::oH + (ee * 9 + q) * A::LP + k] = sGeo[ee * 3 + 0] * ps[0] + sGeo[ee * 3 + 1] * ps[1] + sGeo[ee * 3 + 2] * ps[2];
        // the star matrices' dependence on lambda/rho and mu/rho:
        // Gx[d] = sum_e Theta^{-1}_ed sum_l Kt^e_kl D^{i-1}_lq
        const float gx[3] = {gxi[w * 3], gxi[w * 3 + 1], gxi[w * 3 + 2]};
        // d/d(lam/rho): B^d_{6+d, q<3} = -lam/rho; d/d(mu/rho): B^d_{6+i, sym(i,d)} = -2 mu/rho
        if (q < 3) {
          plr += gx[0] * lv[6] + gx[1] * lv[7] + gx[2] * lv[8];
          pmr += 2.f * (q == 0 ? gx[0] * lv[6] : (q == 1 ? gx[1] * lv[7] : gx[2] * lv[8]));
        } else if (q == 3) {
          pmr += 2.f * (gx[0] * lv[7] + gx[1] * lv[6]);
        } else if (q == 4) {
          pmr += 2.f * (gx[1] * lv[8] + gx[2] * lv[7]);
        } else if (q == 5) {
          pmr += 2.f * (gx[0] * lv[8] + gx[2] * lv[6]);
        }
      }
      __syncthreads();
      // lam D^{i-1}_lq -= sum_e sum_k Kt^e_kl H[e][k][q]
      for (int w = threadIdx.x; w < Lin * 9; w += blockDim.x) {
        const int l = w / 9, q = w - l * 9;
        float s3[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int ee = 0; ee < 3; ++ee) {
          const float* kt = tb + T.KtA + (ee * L + l) * A::LP;
          const float* hq = smem + S::oH + (ee * 9 + q) * A::LP;
#pragma unroll
          for (int kq = 0; kq < Lout / 4; ++kq)
            s3[ee] = dot4(__ldg(reinterpret_cast<const float4*>(kt) + kq), reinterpret_cast<const float4*>(hq)[kq], s3[ee]);
#pragma unroll
          for (int k = Lout / 4 * 4; k < Lout; ++k) s3[ee] = fmaf(__ldg(kt + k), hq[k], s3[ee]);
        }
        lDprev[l * lsp + q] -= s3[0] + s3[1] + s3[2];
      }
      if (i == N) {
        for (int w = threadIdx.x; w < L * 6; w += blockDim.x) {
          const int l = w / 6, p = w - l * 6;
          float s4[4] = {0.f, 0.f, 0.f, 0.f};
          const float* vl = tb + T.VvT + l * A::NQP;
          const float* up = sLu0 + p * A::U0S;
          if constexpr (A::NQP % 4 == 0) {
#pragma unroll 4
            for (int qq = 0; qq < NQ / 4; ++qq)
              s4[qq & 3] = dot4(__ldg(reinterpret_cast<const float4*>(vl) + qq), reinterpret_cast<const float4*>(up)[qq], s4[qq & 3]);
#pragma unroll
            for (int q = NQ / 4 * 4; q < NQ; ++q) s4[0] = fmaf(__ldg(vl + q), up[q], s4[0]);
          } else {
#pragma unroll 8
            for (int q = 0; q < NQ; ++q) s4[q & 3] = fmaf(__ldg(vl + q), up[q], s4[q & 3]);
          }
          sDS[w] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
      }
      __syncthreads();
    }
    block_add(&sRed[6], plr);
    block_add(&sRed[7], pmr);
    block_add(&sRed[0], pxr);
    block_add(&sRed[1], pcr);
    __syncthreads();
    // the cell mean: lambda_eff and mu_eff (and through them cp) at ubar = sqrt(6) Q_0
    if (threadIdx.x == 0) {
      const float r6 = 2.449489742783178f;
      float ub[10];
#pragma unroll
      for (int p = 0; p < 10; ++p) ub[p] = smem[S::oQ + p] * r6;
      const Inv v = invariants(ub);
      // the cp part (cp = sqrt((lambda + 2 mu) / rho)), the boundary fluxes and the CK
      // recursion, in units of lam/rho (d/d(lam/rho) = rho d/dlam)
      const float cp = a.cp[e];
      const float dc = (lam_eff + 2.f * mu_eff > 0.f && cp > 0.f) ? static_cast<float>(sRed[2]) * 0.5f * m.rho_inv / cp : 0.f;
      const double a_lr = (static_cast<double>(dc) + sRed[4]) * m.rho + sRed[6];
      const double a_mr = (static_cast<double>(2.f * dc) + sRed[5]) * m.rho + sRed[7];
      const float al = static_cast<float>(a_lr) * m.rho_inv;   // d/dlambda_eff
      const float am = static_cast<float>(a_mr) * m.rho_inv;   // d/dmu_eff
      const float wv = al * (1.f / 3.f) + 0.5f * am;
      const float ag = ub[9] * m.gamma_r;
#pragma unroll
      for (int p = 0; p < 6; ++p) sLD[p] += r6 * (-ag * wv * v.dxi[p]);
      sLD[9] += r6 * (-m.gamma_r * v.xi * wv + am * m.xi0 * m.gamma_r);
      sRed[0] += static_cast<double>(am * ag);
    }
    __syncthreads();
    for (int w = threadIdx.x; w < A::QS; w += blockDim.x) {
      const int l = w / 10, p = w - 10 * l;
      a.lam_out[e * A::QS + w] = w < L * 10 ? smem[S::oLam + w] + sLD[w] + (p < 6 ? sDS[l * 6 + p] : 0.f) : 0.f;
    }
    if (threadIdx.x == 0) {
      a.g_xi0[e] += sRed[0];
      a.g_cd[e] += sRed[1];
    }
  }
}

}  // namespace adj

template <int N>
cudaError_t launch_adjoint_t(const AdjArgs& a, cudaStream_t s) {
  using SF = adj::FaceSmem<N>;
  using SE = adj::ElemSmem<N>;
  const size_t bf = sizeof(float) * SF::total, be = sizeof(float) * SE::total;
  cudaError_t err = cudaFuncSetAttribute(adj::k_adj_face<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bf));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(adj::k_adj_elem<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(be));
  if (err != cudaSuccess) return err;
  // one CTA per face and per element (the hardware's dynamic scheduling of short CTAs
  // balances the SMs' load to the end of the launch)
  constexpr int64_t kMaxGrid = (int64_t(1) << 31) - 1;
  const int gf = static_cast<int>(a.F < kMaxGrid ? a.F : kMaxGrid);
  const int ge = static_cast<int>(a.E < kMaxGrid ? a.E : kMaxGrid);
  if (gf > 0) adj::k_adj_face<N><<<gf, 128, bf, s>>>(a);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (ge > 0) adj::k_adj_elem<N><<<ge, 128, be, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dg
