// qp_circuit.cuh -- SIMT statevector kernel: embedding, ansatz layers, readout, head,
// Maxwell/energy loss, costates and the adjoint sweep for one group of lanes per point.
//
// Per point the kernel carries four statevectors: phi (the PQC state, Sec. 2.3) and the
// forward-mode tangents phi_x, phi_y, phi_t, whose Pauli-Z bilinears give the exact input
// derivatives of the readout, 2 Re<phi_d|Z_i|phi> (Sec. 2.3 last paragraph: the circuit is
// differentiated w.r.t. its input angles). For the gradient it forms four costates
//   lambda = O phi + sum_d O_d phi_d,   lambda_d = O_d phi,
// with O = sum_i zbar_i Z_i, O_d = sum_i zbar_{d,i} Z_i the loss cotangents of the readout,
// and sweeps the layers backwards: for every single-qubit gate the gradient contribution is
// sum_s Im<lambda_s|P phi_s> for the Pauli generators P, taken after the gate. Rotations of
// the same layer act on different qubits, so all of a layer's contributions can be taken at
// the point after the layer's rotations and before its CNOT ring.
#pragma once
#include <cuda_runtime.h>

#include "qp_common.h"

namespace qpk {

struct SmemLayout {
  int off_gates, off_cenc, off_head, off_eacc, off_hacc, off_loss, off_state, total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// Shared-memory layout of the circuit kernel (identical on host and device).
// head: bytes before the gate table (the schedule; the whole argument block in the
// multi-instance kernel, whose first member is the schedule).
__host__ __device__ inline SmemLayout smem_layout(int n, int L, int m, int nt, int warps,
                                                  int sstride, int ppw, int nE,
                                                  int head = (int)sizeof(QPSched)) {
  SmemLayout s;
  int o = align16(head);
  s.off_gates = o; o = align16(o + L * n * 8 * 4);
  s.off_cenc = o; o = align16(o + n * 4 * 4);
  s.off_head = o; o = align16(o + (3 * m + 3) * 4);
  s.off_eacc = o; o = align16(o + nE * 4);
  s.off_hacc = o; o = align16(o + (3 * m + 3) * 4);
  s.off_loss = o; o = align16(o + (QP_NLP + nt) * 8);
  s.off_state = o; o = align16(o + warps * ppw * sstride * 8);
  s.total = o;
  return s;
}

__device__ __forceinline__ void gate2(float2& x, float2& y, const float* u) {
  const float xr = u[0] * x.x - u[1] * x.y + u[2] * y.x - u[3] * y.y;
  const float xi = u[0] * x.y + u[1] * x.x + u[2] * y.y + u[3] * y.x;
  const float yr = u[4] * x.x - u[5] * x.y + u[6] * y.x - u[7] * y.y;
  const float yi = u[4] * x.y + u[5] * x.x + u[6] * y.y + u[7] * y.x;
  x = make_float2(xr, xi);
  y = make_float2(yr, yi);
}
// Inverse (adjoint) of the same 2x2 gate.
__device__ __forceinline__ void gate2_inv(float2& x, float2& y, const float* u) {
  const float xr = u[0] * x.x + u[1] * x.y + u[4] * y.x + u[5] * y.y;
  const float xi = u[0] * x.y - u[1] * x.x + u[4] * y.y - u[5] * y.x;
  const float yr = u[2] * x.x + u[3] * x.y + u[6] * y.x + u[7] * y.y;
  const float yi = u[2] * x.y - u[3] * x.x + u[6] * y.y - u[7] * y.x;
  x = make_float2(xr, xi);
  y = make_float2(yr, yi);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Unnormalised Walsh-Hadamard transform: out[u] = sum_j (-1)^{popc(u&j)} in[j].
template <int N>
__device__ __forceinline__ void wht(float* v) {
#pragma unroll
  for (int h = 1; h < N; h <<= 1)
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (!(j & h)) {
        const float a = v[j], b = v[j | h];
        v[j] = a + b;
        v[j | h] = a - b;
      }
}
template <int N>
__device__ __forceinline__ float pick(const float* v, int u) {
  float r = v[0];
#pragma unroll
  for (int k = 1; k < N; ++k) r = (u == k) ? v[k] : r;
  return r;
}

// Accumulate sum over pairs of Im<lam|P phi> for P = X, Y, Z on local bit b.
template <int AMPS>
__device__ __forceinline__ void acc_pauli(float* e, const float2* ph, const float2* lm, int b) {
#pragma unroll
  for (int j0 = 0; j0 < AMPS; ++j0) {
    if (j0 & (1 << b)) continue;
    const int j1 = j0 | (1 << b);
    const float2 p0 = ph[j0], p1 = ph[j1], l0 = lm[j0], l1 = lm[j1];
    e[0] += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
    e[1] += (l1.x * p0.x + l1.y * p0.y) - (l0.x * p1.x + l0.y * p1.y);
    e[2] += (l0.x * p0.y - l0.y * p0.x) - (l1.x * p1.y - l1.y * p1.x);
  }
}

template <int GL>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = 1; o < GL; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int GL>
__device__ __forceinline__ float slot_sum(float v) {
#pragma unroll
  for (int o = GL; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Loss terms of one point and their cotangents g = dL/d(Ez,Hx,Hy), gD = dL/d(d field_c/d v_d):
// collocation points carry the residuals of Eqs. 8-10 (1/eps pointwise in the dielectric case,
// Eq. 13 splits res1 by set) and the squared Poynting residual of Eq. 23; IC points the misfit
// of Eq. 17 against the Gaussian pulse of Eq. 14; BC points Ez^2 (PEC). The point's
// contributions to the QP_NLP partial sums go to `lt` (zero where the point adds nothing),
// its energy-slice term of Eq. 31 to `ev` with slice index `slice` (-1: none). The terms are
// FP32 squares of FP32 residuals (one rounding each); callers sum them in FP64 or with
// compensated FP32 sums, so the sums keep the terms' precision (FP64 arithmetic runs at a
// small fraction of the FP32 rate on this part).
__device__ __forceinline__ void point_loss_terms(const QPProblemDev& pb, int set, int64_t pt, int64_t npt,
                                                 const int32_t* counts, float x, float y,
                                                 const float (&f)[3], const float (&D)[3][3], bool active,
                                                 float (&lt)[QP_NLP], int& slice, float& ev,
                                                 float (&g)[3], float (&gD)[3][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g[c] = 0.f;
    gD[c][0] = gD[c][1] = gD[c][2] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < QP_NLP; ++i) lt[i] = 0.f;
  slice = -1;
  ev = 0.f;
  if (!active) return;
  if (set == 0) {
    float eps = 1.f;
    bool diel = false;
    if (pb.medium == 1) {
      const float dx = x - pb.disk_x0, dy = y - pb.disk_y0;
      const float r2 = __fmaf_rn(dx, dx, dy * dy);
      diel = r2 < pb.disk_r * pb.disk_r;
      const float rr = sqrtf(r2);
      eps = 1.f + (pb.eps_r - 1.f) / (1.f + expf(-(pb.disk_r - rr) / pb.sigmoid_w));
    }
    // Eq. 34 (intuitive form): eps = eps_r on the dielectric set, 1 elsewhere, one MSE
    const bool intuitive = pb.medium == 1 && pb.phys_loss == 1;
    const float ie = intuitive ? (diel ? 1.f / pb.eps_r : 1.f) : 1.f / eps;
    const float res1 = D[0][2] - ie * (D[2][0] - D[1][1]);
    const float res2 = D[1][2] + D[0][1];
    const float res3 = D[2][2] - D[0][0];
    const float e = eps * f[0] * D[0][2] + f[1] * D[1][2] + f[2] * D[2][2] -
                    (D[0][0] * f[2] + f[0] * D[2][0]) + (D[0][1] * f[1] + f[0] * D[1][1]);
    const float N = (float)(pb.norm[0] > 0 ? pb.norm[0] : npt);
    float N1 = N;
    if (pb.medium == 1 && !intuitive) {
      const float nd = (float)(pb.norm[0] > 0 ? pb.norm_diel : counts[0]);
      N1 = diel ? nd : N - nd;
    }
    const float k1 = 2.f * res1 / N1, k2 = 2.f * res2 / N, k3 = 2.f * res3 / N;
    const float kE = 2.f * pb.w_energy * e / N;
    g[0] = kE * (eps * D[0][2] - D[2][0] + D[1][1]);
    g[1] = kE * (D[1][2] + D[0][1]);
    g[2] = kE * (D[2][2] - D[0][0]);
    gD[0][0] = -k3 - kE * f[2];
    gD[0][1] = k2 + kE * f[1];
    gD[0][2] = k1 + kE * eps * f[0];
    gD[1][1] = k1 * ie + kE * f[0];
    gD[1][2] = k2 + kE * f[1];
    gD[2][0] = -k1 * ie - kE * f[0];
    gD[2][2] = k3 + kE * f[2];
    const float r1sq = res1 * res1;
    lt[0] = diel && !intuitive ? 0.f : r1sq;
    lt[1] = diel && !intuitive ? r1sq : 0.f;
    lt[2] = res2 * res2;
    lt[3] = res3 * res3;
    lt[4] = e * e;
    if (pb.energy_nt > 0 && pb.energy_slice > 0) {
      const int64_t k = (pt + pb.colloc_off) / pb.energy_slice;
      if (k < pb.energy_nt) {
        slice = (int)k;
        ev = 0.5f * (eps * f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
      }
    }
  } else if (set == 1) {
    const float dx = x - pb.ic_x0, dy = y - pb.ic_y0;
    const float e0 = expf(-(dx * dx + dy * dy) / (2.f * pb.ic_sigma * pb.ic_sigma));
    const float k = 2.f * pb.w_ic / (float)(pb.norm[1] > 0 ? pb.norm[1] : npt);
    g[0] = k * (f[0] - e0);
    g[1] = k * f[1];
    g[2] = k * f[2];
    const float d0 = f[0] - e0;
    lt[5] = d0 * d0 + f[1] * f[1] + f[2] * f[2];
  } else {
    g[0] = 2.f * pb.w_bc * f[0] / (float)(pb.norm[2] > 0 ? pb.norm[2] : npt);
    lt[6] = f[0] * f[0];
  }
}

// point_loss_terms with the partial sums added to `loss` (shared FP64 partials, only when `acc`).
__device__ __forceinline__ void point_loss(const QPProblemDev& pb, int set, int64_t pt, int64_t npt,
                                           const int32_t* counts, float x, float y,
                                           const float (&f)[3], const float (&D)[3][3], bool active,
                                           bool acc, double* loss, float (&g)[3], float (&gD)[3][3]) {
  float lt[QP_NLP], ev;
  int slice;
  point_loss_terms(pb, set, pt, npt, counts, x, y, f, D, active, lt, slice, ev, g, gD);
  if (active && acc) {
    if (set == 0) {
      atomicAdd(&loss[lt[1] != 0.f ? 1 : 0], (double)(lt[0] + lt[1]));
      atomicAdd(&loss[2], (double)lt[2]);
      atomicAdd(&loss[3], (double)lt[3]);
      atomicAdd(&loss[4], (double)lt[4]);
      if (slice >= 0) atomicAdd(&loss[QP_NLP + slice], (double)ev);
    } else if (set == 1) {
      atomicAdd(&loss[5], (double)lt[5]);
    } else {
      atomicAdd(&loss[6], (double)lt[6]);
    }
  }
}

struct Shared {
  const QPSched* s;
  const float* gates;
  const float* cenc;
  const float* head;
  float* eacc;
  float* hacc;
  double* loss;
};

// Gate matrices of the pass's gate qubits (uniform shared-memory reads).
template <int LB>
__device__ __forceinline__ void load_gates(const Shared& sh, const QPSched& S, int l, int n, int P,
                                           int ng, float (&U)[LB][8]) {
#pragma unroll
  for (int b = 0; b < LB; ++b) {
    if (b < ng) {
      const float4* g = reinterpret_cast<const float4*>(sh.gates + (l * n + S.ql[P][b]) * 8);
      const float4 u0 = g[0], u1 = g[1];
      U[b][0] = u0.x; U[b][1] = u0.y; U[b][2] = u0.z; U[b][3] = u0.w;
      U[b][4] = u1.x; U[b][5] = u1.y; U[b][6] = u1.z; U[b][7] = u1.w;
    }
  }
}

// Embedding factor of one local qubit: G(theta)|0> and d/dtheta of it, basis 0 and 1.
struct EmbedLocal {
  float2 g0, g1, h0, h1;
  float J[3];
};
__device__ __forceinline__ void embed_factor(int enc, float c, float s, int bit, float2& gv,
                                             float2& gd) {
  if (enc == 0) {  // RX|0> = (c, -i s); d/dtheta = (-s/2, -i c/2)
    gv = bit ? make_float2(0.f, -s) : make_float2(c, 0.f);
    gd = bit ? make_float2(0.f, -0.5f * c) : make_float2(-0.5f * s, 0.f);
  } else {         // RY|0> = (c, s); d/dtheta = (-s/2, c/2)
    gv = bit ? make_float2(s, 0.f) : make_float2(c, 0.f);
    gd = bit ? make_float2(0.5f * c, 0.f) : make_float2(-0.5f * s, 0.f);
  }
}
__device__ __forceinline__ float pick3(const float4& t, int d) {
  return d == 0 ? t.y : (d == 1 ? t.z : t.w);
}

// One warp-task: PPW points of one set. nv = 4 statevectors per point (phi and the tangents
// phi_x, phi_y, phi_t) for collocation points, 1 where only the fields are needed. Every hot
// loop body handles one vector (forward) or one (state, costate) pair (adjoint), so the code
// that runs per gate pass stays small.
template <int NQ, bool GRAD, bool CRZ>
__device__ __forceinline__ void run_task(const QPCircArgs& a, const Shared& sh, float2* wstate,
                                         int set, int64_t first_pt, int lane, int nv) {
  using Gm = QPGeo<NQ>;
  constexpr int LB = Gm::LB, AMPS = Gm::AMPS, GL = Gm::GL, DIM = Gm::DIM;
  const QPSched& S = *sh.s;
  const int n = a.n, L = a.L, m = a.m, npl = S.npl;
  const int slot = lane / GL;
  const int lin = lane % GL;
  const int64_t npt = a.npts[set];
  const int64_t pt = first_pt + slot;
  const bool active = pt < npt;
  const int64_t ptc = active ? pt : npt - 1;
  const int64_t gp = a.pt_base[set] + ptc;
  float2* st = wstate + slot * a.sstride;
  const float4* tj = reinterpret_cast<const float4*>(a.thetaJ) + gp * n;
  int ad[AMPS];

  // ------------------------------------------------------------------ forward passes
  for (int l = 0; l < L; ++l) {
    for (int p = 0; p < npl; ++p) {
      const int P = l * npl + p;
      const int la = S.lane_addr[P][lane];
#pragma unroll
      for (int j = 0; j < AMPS; ++j) ad[j] = la ^ S.joff[P][j];
      const int ng = S.ngate[P];
      float U[LB][8];
      load_gates<LB>(sh, S, l, n, P, ng, U);
      // CRZ mesh (Eq. 29) after the last rotation pass of the layer: one phase per amplitude,
      // looked up by its logical basis index (the frame is the identity: no CNOTs)
      const bool crz_here = CRZ && p == npl - 1;
      float2 dph[AMPS];
      if (crz_here) {
        const int kb = S.klog[l][lane];
#pragma unroll
        for (int j = 0; j < AMPS; ++j) dph[j] = __ldg(&a.crz[l * DIM + (kb ^ S.jlog[l][j])]);
      }
      EmbedLocal el[LB];
      uint32_t localmask = 0;
      if (P == 0) {
#pragma unroll
        for (int b = 0; b < LB; ++b) {
          const int q = S.ql[0][b];
          localmask |= 1u << q;
          const float4 t = tj[q];
          float sn, cs;
          sincosf(0.5f * t.x, &sn, &cs);
          embed_factor(a.enc, cs, sn, 0, el[b].g0, el[b].h0);
          embed_factor(a.enc, cs, sn, 1, el[b].g1, el[b].h1);
          el[b].J[0] = t.y; el[b].J[1] = t.z; el[b].J[2] = t.w;
        }
      }
#pragma unroll 1
      for (int v = 0; v < nv; ++v) {
        float2 r[AMPS];
        float2* sv = st + v * DIM;
        if (P == 0) {
          // product state G(theta_q)|0> over all qubits, or its tangent in direction d = v-1:
          // psi_d = sum_q J_qd dpsi/dtheta_q, by the product rule (no division)
          const int d = v - 1;
          const uint32_t K = S.enc_k[lane];
          float2 A = make_float2(1.f, 0.f), Ad = make_float2(0.f, 0.f);
          for (int q = 0; q < n; ++q) {
            if ((localmask >> q) & 1u) continue;
            const float4 t = tj[q];
            float sn, cs;
            sincosf(0.5f * t.x, &sn, &cs);
            float2 gv, gd;
            embed_factor(a.enc, cs, sn, (K >> (n - 1 - q)) & 1, gv, gd);
            if (v > 0) Ad = cadd(cmul(Ad, gv), cscale(cmul(A, gd), pick3(t, d)));
            A = cmul(A, gv);
          }
#pragma unroll
          for (int j = 0; j < AMPS; ++j) {
            float2 B = make_float2(1.f, 0.f), Bd = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < LB; ++b) {
              const bool bit = (j >> b) & 1;
              const float2 gv = bit ? el[b].g1 : el[b].g0;
              if (v > 0) {
                const float2 gd = bit ? el[b].h1 : el[b].h0;
                const float Jb = d == 0 ? el[b].J[0] : (d == 1 ? el[b].J[1] : el[b].J[2]);
                Bd = cadd(cmul(Bd, gv), cscale(cmul(B, gd), Jb));
              }
              B = cmul(B, gv);
            }
            r[j] = v > 0 ? cadd(cmul(Ad, B), cmul(A, Bd)) : cmul(A, B);
          }
        } else {
#pragma unroll
          for (int j = 0; j < AMPS; ++j) r[j] = sv[ad[j]];
        }
#pragma unroll
        for (int b = 0; b < LB; ++b)
          if (b < ng)
#pragma unroll
            for (int j0 = 0; j0 < AMPS; ++j0)
              if (!(j0 & (1 << b))) gate2(r[j0], r[j0 | (1 << b)], U[b]);
        if (crz_here) {
#pragma unroll
          for (int j = 0; j < AMPS; ++j) r[j] = cmul(r[j], dph[j]);
        }
#pragma unroll
        for (int j = 0; j < AMPS; ++j) sv[ad[j]] = r[j];
      }
      __syncwarp();
    }
  }

  // ------------------------------------------------------------------ readout (Sec. 2.3)
  // In the last pass's view: z_i = sum_k |phi_k|^2 s_i(k) with the lane's sign and the
  // Walsh index of Z_i over the local bits, s_i(k_j) = sigma_i (-1)^{popc(sel_i & j)};
  // d z_i / d v_d = 2 Re <phi_d|Z_i|phi>.
  float wv[4][AMPS];
#pragma unroll
  for (int j = 0; j < AMPS; ++j) {
    const float2 ph = st[ad[j]];
    wv[0][j] = ph.x * ph.x + ph.y * ph.y;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float q = 0.f;
      if (nv == 4) {
        const float2 pd = st[(1 + d) * DIM + ad[j]];
        q = 2.f * (pd.x * ph.x + pd.y * ph.y);
      }
      wv[1 + d][j] = q;
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) wht<AMPS>(wv[v]);
  const uint32_t rmask = S.ro_mask[lane];
  float z[QP_MAXQ], dz[3][QP_MAXQ];
#pragma unroll
  for (int i = 0; i < QP_MAXQ; ++i) {
    if (i < m) {
      const int u = S.ro_sel[i];
      const float sg = ((rmask >> i) & 1u) ? -1.f : 1.f;
      z[i] = group_sum<GL>(sg * pick<AMPS>(wv[0], u));
#pragma unroll
      for (int d = 0; d < 3; ++d)
        dz[d][i] = nv == 4 ? group_sum<GL>(sg * pick<AMPS>(wv[1 + d], u)) : 0.f;
    } else {
      z[i] = 0.f;
      dz[0][i] = dz[1][i] = dz[2][i] = 0.f;
    }
  }
  // ------------------------------------------------------------------ linear head
  float f[3], D[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float acc = sh.head[3 * m + c];
    float ad3[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i)
      if (i < m) {
        const float w = sh.head[c * m + i];
        acc += w * z[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) ad3[d] += w * dz[d][i];
      }
    f[c] = acc;
#pragma unroll
    for (int d = 0; d < 3; ++d) D[c][d] = ad3[d];
  }
  if (!GRAD) {
    if (active && lin == 0) {
      const int64_t go = a.pt_base[set] + pt;   // global point index (set 0 alone: pt)
#pragma unroll
      for (int c = 0; c < 3; ++c) a.out_f[go * 3 + c] = f[c];
      if (nv == 4 && a.out_df) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) a.out_df[go * 9 + c * 3 + d] = D[c][d];
      }
    }
    return;
  }
  // ------------------------------------------------------------------ loss and cotangents
  const float* xp = a.pts[set] + ptc * 3;
  float g[3], gD[3][3];
  // rows of set 2 past the boundary points carry given cotangents (mirrored points of L_sym)
  const bool given = set == 2 && pt >= a.nbc;
  point_loss(a.pb, set, pt, set == 2 ? a.nbc : npt, a.counts, xp[0], xp[1], f, D, active && !given,
             lin == 0, sh.loss, g, gD);
  if (given && active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] = a.gext[(pt - a.nbc) * 3 + c];
  }
  if (set == 0 && a.gsym && active) {
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] += a.gsym[pt * 3 + c];
  }
  // back through the head: zbar = W^T g, zbar_d = W^T g_d; head gradients
  float zb[QP_MAXQ], zbd[3][QP_MAXQ];
#pragma unroll
  for (int i = 0; i < QP_MAXQ; ++i) {
    zb[i] = 0.f;
    zbd[0][i] = zbd[1][i] = zbd[2][i] = 0.f;
    if (i < m) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float w = sh.head[c * m + i];
        zb[i] += w * g[c];
#pragma unroll
        for (int d = 0; d < 3; ++d) zbd[d][i] += w * gD[c][d];
      }
    }
  }
  if (active && lin == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i)
        if (i < m)
          atomicAdd(&sh.hacc[c * m + i],
                    g[c] * z[i] + gD[c][0] * dz[0][i] + gD[c][1] * dz[1][i] + gD[c][2] * dz[2][i]);
      atomicAdd(&sh.hacc[3 * m + c], g[c]);
    }
  }
  // ------------------------------------------------------------------ costates
  // O_j = sum_i zbar_i s_i(k_j) = WHT(h)[j], h[u] = sum_{i: sel_i = u} sigma_i zbar_i.
  float Ov[4][AMPS];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int u = 0; u < AMPS; ++u) Ov[v][u] = 0.f;
#pragma unroll
  for (int i = 0; i < QP_MAXQ; ++i) {
    if (i < m) {
      const int u0 = S.ro_sel[i];
      const float sg = ((rmask >> i) & 1u) ? -1.f : 1.f;
#pragma unroll
      for (int u = 0; u < AMPS; ++u) {
        const float hit = (u == u0) ? sg : 0.f;
        Ov[0][u] += hit * zb[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) Ov[1 + d][u] += hit * zbd[d][i];
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) wht<AMPS>(Ov[v]);
  // lambda = O phi + sum_d O_d phi_d (slot nv), lambda_d = O_d phi (slots nv + 1 + d)
#pragma unroll
  for (int j = 0; j < AMPS; ++j) {
    const float2 ph = st[ad[j]];
    float2 lam = cscale(ph, Ov[0][j]);
    if (nv == 4) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        lam = cadd(lam, cscale(st[(1 + d) * DIM + ad[j]], Ov[1 + d][j]));
        st[(5 + d) * DIM + ad[j]] = cscale(ph, Ov[1 + d][j]);
      }
    }
    st[nv * DIM + ad[j]] = lam;
  }
  __syncwarp();

  // ------------------------------------------------------------------ adjoint sweep
  const bool wdt = a.want_dtheta && nv == 4;
  for (int l = L - 1; l >= 0; --l) {
    for (int p = npl - 1; p >= 0; --p) {
      const int P = l * npl + p;
      const int la = S.lane_addr[P][lane];
#pragma unroll
      for (int j = 0; j < AMPS; ++j) ad[j] = la ^ S.joff[P][j];
      const int ng = S.ngate[P];
      float U[LB][8];
      load_gates<LB>(sh, S, l, n, P, ng, U);
      float E[LB][3];
#pragma unroll
      for (int b = 0; b < LB; ++b) E[b][0] = E[b][1] = E[b][2] = 0.f;
      // CRZ mesh of this layer (its last pass): the gradient sums w(k) = sum_s Im(lambda_s(k)^*
      // phi_s(k)) are taken after the mesh, then the mesh is undone on states and costates
      const bool crz_here = CRZ && p == npl - 1;
      float2 dph[AMPS];
      float wk[AMPS];
#pragma unroll
      for (int j = 0; j < AMPS; ++j) wk[j] = 0.f;
      if (crz_here) {
        const int kb = S.klog[l][lane];
#pragma unroll
        for (int j = 0; j < AMPS; ++j) {
          const float2 d = __ldg(&a.crz[l * DIM + (kb ^ S.jlog[l][j])]);
          dph[j] = make_float2(d.x, -d.y);
        }
      }
      // (state, costate) pairs: vector s and vector nv + s
#pragma unroll 1
      for (int s = 0; s < nv; ++s) {
        float2 xs[AMPS], ys[AMPS];
        float2* sx = st + s * DIM;
        float2* sy = st + (nv + s) * DIM;
#pragma unroll
        for (int j = 0; j < AMPS; ++j) {
          xs[j] = sx[ad[j]];
          ys[j] = sy[ad[j]];
        }
        if (crz_here) {
#pragma unroll
          for (int j = 0; j < AMPS; ++j) {
            wk[j] += ys[j].x * xs[j].y - ys[j].y * xs[j].x;
            xs[j] = cmul(xs[j], dph[j]);
            ys[j] = cmul(ys[j], dph[j]);
          }
        }
#pragma unroll
        for (int b = 0; b < LB; ++b)
          if (b < ng) acc_pauli<AMPS>(E[b], xs, ys, b);
        if (l > 0) {
#pragma unroll
          for (int b = 0; b < LB; ++b)
            if (b < ng)
#pragma unroll
              for (int j0 = 0; j0 < AMPS; ++j0)
                if (!(j0 & (1 << b))) {
                  gate2_inv(xs[j0], xs[j0 | (1 << b)], U[b]);
                  gate2_inv(ys[j0], ys[j0 | (1 << b)], U[b]);
                }
        }
        if (l > 0 || crz_here) {
#pragma unroll
          for (int j = 0; j < AMPS; ++j) {
            sx[ad[j]] = xs[j];
            sy[ad[j]] = ys[j];
          }
        }
      }
      if (crz_here) {
        // Z-correlation sums of the layer: Z_t = sum_k w(k) z_t(k) and Z_ct = sum_k w(k) z_c(k)
        // z_t(k), z_q(k) = 1 - 2 b_q(k); lanes of a point hold disjoint k = K | sv_j
        const int kb = S.klog[l][lane];
        float* zacc = sh.eacc + 3 * NQ * L + l * qp_crz_sums(a.ansatz, NQ);
#pragma unroll
        for (int t = 0; t < NQ; ++t) {
          float zt = 0.f;
#pragma unroll
          for (int j = 0; j < AMPS; ++j) {
            const int kj = kb ^ S.jlog[l][j];
            zt += ((kj >> (NQ - 1 - t)) & 1) ? -wk[j] : wk[j];
          }
          zt = slot_sum<GL>(group_sum<GL>(zt));
          if (lane == 0) atomicAdd(&zacc[t], zt);
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c)
#pragma unroll
          for (int t = c + 1; t < NQ; ++t) {
            float zct = 0.f;
#pragma unroll
            for (int j = 0; j < AMPS; ++j) {
              const int kj = kb ^ S.jlog[l][j];
              const int par = ((kj >> (NQ - 1 - t)) ^ (kj >> (NQ - 1 - c))) & 1;
              zct += par ? -wk[j] : wk[j];
            }
            zct = slot_sum<GL>(group_sum<GL>(zct));
            if (lane == 0) atomicAdd(&zacc[NQ + qp_pair_index(NQ, c, t)], zct);
          }
      }
      float E2[LB][3][3];  // layer 0: Im<lambda_d|P phi> for the input-Jacobian gradient
#pragma unroll
      for (int b = 0; b < LB; ++b)
#pragma unroll
        for (int k = 0; k < 3; ++k) E2[b][0][k] = E2[b][1][k] = E2[b][2][k] = 0.f;
      if (l == 0 && wdt) {
        float2 ph[AMPS];
#pragma unroll
        for (int j = 0; j < AMPS; ++j) ph[j] = st[ad[j]];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float2 lm[AMPS];
#pragma unroll
          for (int j = 0; j < AMPS; ++j) lm[j] = st[(5 + d) * DIM + ad[j]];
#pragma unroll
          for (int b = 0; b < LB; ++b)
            if (b < ng) acc_pauli<AMPS>(E2[b][d], ph, lm, b);
        }
      }
      __syncwarp();
      // reductions: per point for layer 0 (embedding gradients), then over the warp
#pragma unroll
      for (int b = 0; b < LB; ++b) {
        if (b >= ng) continue;
        const int q = S.ql[P][b];
        if (l == 0) {
          float e3[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) e3[k] = group_sum<GL>(E[b][k]);
          if (a.want_dtheta) {
            const float c0 = sh.cenc[q * 4 + 0], c1 = sh.cenc[q * 4 + 1], c2 = sh.cenc[q * 4 + 2];
            float outv[4];
            outv[0] = c0 * e3[0] + c1 * e3[1] + c2 * e3[2];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const float s0 = group_sum<GL>(E2[b][d][0]);
              const float s1 = group_sum<GL>(E2[b][d][1]);
              const float s2 = group_sum<GL>(E2[b][d][2]);
              outv[1 + d] = c0 * s0 + c1 * s1 + c2 * s2;
            }
            if (active && lin == 0)
              reinterpret_cast<float4*>(a.dthetaJ)[gp * n + q] =
                  make_float4(outv[0], outv[1], outv[2], outv[3]);
          }
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float t = slot_sum<GL>(e3[k]);
            if (lane == 0) atomicAdd(&sh.eacc[(l * n + q) * 3 + k], t);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float t = slot_sum<GL>(group_sum<GL>(E[b][k]));
            if (lane == 0) atomicAdd(&sh.eacc[(l * n + q) * 3 + k], t);
          }
        }
      }
    }
  }
}

// Persistent kernel: every warp takes warp-tasks (PPW points of one set) in turn; block
// partials of the loss sums and gradient sums are written at the end. CRZ: the ansatz has a
// CRZ mesh (compiled apart, so the other ansatze carry none of its registers).
template <int NQ, bool GRAD, bool CRZ>
__global__ void __launch_bounds__(384) circuit_kernel(const __grid_constant__ QPCircArgs a) {
  using Gm = QPGeo<NQ>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = GRAD ? a.pb.energy_nt : 0;
  const SmemLayout lay = smem_layout(a.n, a.L, a.m, nt, warps, a.sstride, Gm::PPW, a.nE);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&a.s);
    uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(QPSched) / 4); i += blockDim.x) dst[i] = src[i];
    float* g = reinterpret_cast<float*>(smem + lay.off_gates);
    for (int i = threadIdx.x; i < a.L * a.n * 8; i += blockDim.x) g[i] = a.gates[i];
    float* c = reinterpret_cast<float*>(smem + lay.off_cenc);
    for (int i = threadIdx.x; i < a.n * 4; i += blockDim.x) c[i] = a.cenc ? a.cenc[i] : 0.f;
    float* h = reinterpret_cast<float*>(smem + lay.off_head);
    for (int i = threadIdx.x; i < 3 * a.m + 3; i += blockDim.x) h[i] = a.head[i];
    float* e = reinterpret_cast<float*>(smem + lay.off_eacc);
    for (int i = threadIdx.x; i < a.nE; i += blockDim.x) e[i] = 0.f;
    float* ha = reinterpret_cast<float*>(smem + lay.off_hacc);
    for (int i = threadIdx.x; i < 3 * a.m + 3; i += blockDim.x) ha[i] = 0.f;
    double* lo = reinterpret_cast<double*>(smem + lay.off_loss);
    for (int i = threadIdx.x; i < QP_NLP + nt; i += blockDim.x) lo[i] = 0.0;
  }
  __syncthreads();
  Shared sh;
  sh.s = reinterpret_cast<const QPSched*>(smem);
  sh.gates = reinterpret_cast<const float*>(smem + lay.off_gates);
  sh.cenc = reinterpret_cast<const float*>(smem + lay.off_cenc);
  sh.head = reinterpret_cast<const float*>(smem + lay.off_head);
  sh.eacc = reinterpret_cast<float*>(smem + lay.off_eacc);
  sh.hacc = reinterpret_cast<float*>(smem + lay.off_hacc);
  sh.loss = reinterpret_cast<double*>(smem + lay.off_loss);
  float2* wstate = reinterpret_cast<float2*>(smem + lay.off_state) + warp * Gm::PPW * a.sstride;

  const int64_t total = a.task_end[2];
  const int64_t stride = (int64_t)gridDim.x * warps;
  for (int64_t t = (int64_t)blockIdx.x * warps + warp; t < total; t += stride) {
    int set = 0;
    int64_t base = 0;
    if (t >= a.task_end[0]) { set = 1; base = a.task_end[0]; }
    if (t >= a.task_end[1]) { set = 2; base = a.task_end[1]; }
    const int64_t first = (t - base) * Gm::PPW;
    const int nv = (set == 0 && (GRAD || a.want_df)) ? 4 : 1;
    run_task<NQ, GRAD, CRZ>(a, sh, wstate, set, first, lane, nv);
  }
  if (!GRAD) return;
  __syncthreads();
  double* bl = a.blk_loss + (int64_t)blockIdx.x * a.loss_stride;
  for (int i = threadIdx.x; i < QP_NLP + nt; i += blockDim.x) bl[i] = sh.loss[i];
  float* bg = a.blk_grad + (int64_t)blockIdx.x * a.grad_stride;
  for (int i = threadIdx.x; i < a.nE; i += blockDim.x) bg[i] = sh.eacc[i];
  for (int i = threadIdx.x; i < 3 * a.m + 3; i += blockDim.x) bg[a.nE + i] = sh.hacc[i];
}

// ------------------------------------------------------------------------- multi-instance launch
// Independent loss evaluations (instances: each its own circuit, problem, parameters and point
// sets) of one qubit count in one persistent launch. Instance i's warp-tasks are cut into items of
// tasks_per_item[i] consecutive tasks; a CTA takes the next item from one atomic counter,
// loads the instance's argument block (schedule included), gate table and head into shared
// memory when the instance changes, runs the item's tasks on its warps and writes the item's
// loss and gradient partials to slot (item - first item of the instance) of the instance's
// block partials, so the instance's reduction sums exactly its items. Items are handed out in
// increasing order, so a CTA meets every instance in one run of consecutive items.
#define QP_MULTI_MAX 64
struct QPMultiArgs {
  int32_t count;                              // instances of this launch (<= QP_MULTI_MAX)
  unsigned long long* queue;                  // item counter, zero before the launch
  const QPCircArgs* desc[QP_MULTI_MAX];       // argument block of each instance (device memory)
  int64_t item_end[QP_MULTI_MAX];             // cumulative item counts
  int32_t tasks_per_item[QP_MULTI_MAX];
};

// The argument block of one instance into device memory (and the item counter zeroed).
__global__ void store_desc_kernel(const __grid_constant__ QPCircArgs a, QPCircArgs* dst,
                                  unsigned long long* queue) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&a);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(QPCircArgs) / 4); i += blockDim.x) d[i] = src[i];
  if (queue && threadIdx.x == 0) *queue = 0ull;
}

template <int NQ, bool CRZ>
__device__ __forceinline__ void multi_tasks(const QPCircArgs& a, const Shared& sh, unsigned char* state,
                                            int64_t t0, int64_t t1, int warp, int warps, int lane) {
  using Gm = QPGeo<NQ>;
  float2* wstate = reinterpret_cast<float2*>(state) + warp * Gm::PPW * a.sstride;
  for (int64_t t = t0 + warp; t < t1; t += warps) {
    int set = 0;
    int64_t base = 0;
    if (t >= a.task_end[0]) { set = 1; base = a.task_end[0]; }
    if (t >= a.task_end[1]) { set = 2; base = a.task_end[1]; }
    run_task<NQ, true, CRZ>(a, sh, wstate, set, (t - base) * Gm::PPW, lane, set == 0 ? 4 : 1);
  }
}

// One qubit count per kernel: the register allocation of the single-instance kernel (a switch
// over several counts in one kernel is allocated for all of them at once and spills).
template <int NQ, bool CRZ>
__global__ void __launch_bounds__(384) circuit_multi_kernel(const __grid_constant__ QPMultiArgs m) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  QPCircArgs& A = *reinterpret_cast<QPCircArgs*>(smem);
  const int warps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = m.item_end[m.count - 1];
  int cur = -1;
  SmemLayout lay{};
  Shared sh{};
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(m.queue, 1ull);
    __syncthreads();
    const int64_t item = s_item;
    if (item >= total) break;
    int i = 0;
    while (m.item_end[i] <= item) ++i;
    const int64_t ib = i > 0 ? m.item_end[i - 1] : 0;
    if (i != cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(m.desc[i]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
      for (int k = threadIdx.x; k < (int)(sizeof(QPCircArgs) / 4); k += blockDim.x) dst[k] = __ldg(src + k);
      __syncthreads();
      const int n = NQ;
      lay = smem_layout(n, A.L, A.m, A.pb.energy_nt, warps, A.sstride, QPGeo<NQ>::PPW, A.nE, (int)sizeof(QPCircArgs));
      float* g = reinterpret_cast<float*>(smem + lay.off_gates);
      for (int k = threadIdx.x; k < A.L * n * 8; k += blockDim.x) g[k] = A.gates[k];
      float* c = reinterpret_cast<float*>(smem + lay.off_cenc);
      for (int k = threadIdx.x; k < n * 4; k += blockDim.x) c[k] = A.cenc ? A.cenc[k] : 0.f;
      float* h = reinterpret_cast<float*>(smem + lay.off_head);
      for (int k = threadIdx.x; k < 3 * A.m + 3; k += blockDim.x) h[k] = A.head[k];
      sh.s = &A.s;
      sh.gates = g;
      sh.cenc = c;
      sh.head = h;
      sh.eacc = reinterpret_cast<float*>(smem + lay.off_eacc);
      sh.hacc = reinterpret_cast<float*>(smem + lay.off_hacc);
      sh.loss = reinterpret_cast<double*>(smem + lay.off_loss);
      cur = i;
    }
    const int nt = A.pb.energy_nt;
    for (int k = threadIdx.x; k < A.nE; k += blockDim.x) sh.eacc[k] = 0.f;
    for (int k = threadIdx.x; k < 3 * A.m + 3; k += blockDim.x) sh.hacc[k] = 0.f;
    for (int k = threadIdx.x; k < QP_NLP + nt; k += blockDim.x) sh.loss[k] = 0.0;
    __syncthreads();
    const int64_t ntask = A.task_end[2];
    const int64_t t0 = (item - ib) * m.tasks_per_item[i];
    const int64_t t1 = t0 + m.tasks_per_item[i] < ntask ? t0 + m.tasks_per_item[i] : ntask;
    multi_tasks<NQ, CRZ>(A, sh, smem + lay.off_state, t0, t1, warp, warps, lane);
    __syncthreads();
    const int64_t slot = item - ib;
    double* bl = A.blk_loss + slot * A.loss_stride;
    for (int k = threadIdx.x; k < QP_NLP + nt; k += blockDim.x) bl[k] = sh.loss[k];
    float* bg = A.blk_grad + slot * A.grad_stride;
    for (int k = threadIdx.x; k < A.nE; k += blockDim.x) bg[k] = sh.eacc[k];
    for (int k = threadIdx.x; k < 3 * A.m + 3; k += blockDim.x) bg[A.nE + k] = sh.hacc[k];
  }
}

}  // namespace qpk
