// qp_aux.cuh -- kernels around the circuit: gate preparation, premap forward/backward,
// weight-gradient reduction and the final FP64 reduction of loss terms and gradients.
#pragma once
#include <cuda_runtime.h>

#include "qp_common.h"

namespace qpk {

struct PrepArgs {
  const float* params;
  int64_t circ_off;
  int32_t n, L, ansatz, enc;
  float* gates;   // [L][n][8]
  float* cmat;    // [L][n][3][4]: d loss / d angle_k = sum_Q cmat[k][Q] E_Q
  float* cenc;    // [n][4]
  int32_t* counts;
  int32_t* status;
};

struct dc { double x, y; };
__device__ inline dc dmul(dc a, dc b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ inline dc dadd(dc a, dc b) { return {a.x + b.x, a.y + b.y}; }
__device__ inline dc dconj(dc a) { return {a.x, -a.y}; }
struct M2 { dc a, b, c, d; };
__device__ inline M2 mmul(const M2& p, const M2& q) {
  return {dadd(dmul(p.a, q.a), dmul(p.b, q.c)), dadd(dmul(p.a, q.b), dmul(p.b, q.d)),
          dadd(dmul(p.c, q.a), dmul(p.d, q.c)), dadd(dmul(p.c, q.b), dmul(p.d, q.d))};
}
__device__ inline M2 mdag(const M2& p) { return {dconj(p.a), dconj(p.c), dconj(p.b), dconj(p.d)}; }
__device__ inline M2 m_rz(double t) {
  double s, c;
  sincos(0.5 * t, &s, &c);
  return {{c, -s}, {0, 0}, {0, 0}, {c, s}};
}
__device__ inline M2 m_ry(double t) {
  double s, c;
  sincos(0.5 * t, &s, &c);
  return {{c, 0}, {-s, 0}, {s, 0}, {c, 0}};
}
__device__ inline M2 m_rx(double t) {
  double s, c;
  sincos(0.5 * t, &s, &c);
  return {{c, 0}, {0, -s}, {0, -s}, {c, 0}};
}
__device__ inline M2 m_pauli(int k) {
  if (k == 0) return {{0, 0}, {1, 0}, {1, 0}, {0, 0}};
  if (k == 1) return {{0, 0}, {0, -1}, {0, 1}, {0, 0}};
  return {{1, 0}, {0, 0}, {0, 0}, {-1, 0}};
}
// c_Q = Tr(Q V G V^dag) / 2 for Q = X, Y, Z: coordinates of the conjugated generator.
__device__ inline void pauli_coords(const M2& V, int G, float* out) {
  const M2 M = mmul(mmul(V, m_pauli(G)), mdag(V));
  out[0] = (float)(0.5 * (M.c.x + M.b.x));  // Tr(X M) = M10 + M01
  out[1] = (float)(0.5 * (M.c.y - M.b.y));  // Tr(Y M) = -i M10 + i M01 (real part)
  out[2] = (float)(0.5 * (M.a.x - M.d.x));  // Tr(Z M) = M00 - M11
  out[3] = 0.f;
}

// One thread per (layer, qubit): forward gate matrix and gradient coordinates.
__global__ void prep_kernel(PrepArgs a) {
  const int t = threadIdx.x + blockIdx.x * blockDim.x;
  // status word, dielectric count and the two operand-range maxima of the FP16 contractions
  if (t == 0) { a.counts[0] = 0; a.status[0] = 0; a.status[16] = 0; a.status[17] = 0; }
  if (t >= a.L * a.n) return;
  const int l = t / a.n, q = t % a.n;
  const int k = qp_ansatz_k(a.ansatz);
  const float* p = a.params + a.circ_off + (int64_t)l * qp_layer_params(a.ansatz, a.n) + (int64_t)q * k;
  M2 U, Vk[3];
  int Gk[3];
  const M2 I2 = {{1, 0}, {0, 0}, {0, 0}, {1, 0}};
  if (a.ansatz == 0) {  // RY(a) then RZ(b): U = RZ(b) RY(a)
    const M2 rz = m_rz(p[1]), ry = m_ry(p[0]);
    U = mmul(rz, ry);
    Vk[0] = rz; Gk[0] = 1;
    Vk[1] = I2; Gk[1] = 2;
  } else if (a.ansatz == 4) {  // RX(a) (Cross-Mesh)
    U = m_rx(p[0]);
    Vk[0] = I2; Gk[0] = 0;
  } else if (a.ansatz == 5) {  // RX(a) then RZ(b): U = RZ(b) RX(a) (Cross-Mesh-2-Rotations)
    const M2 rz = m_rz(p[1]);
    U = mmul(rz, m_rx(p[0]));
    Vk[0] = rz; Gk[0] = 0;
    Vk[1] = I2; Gk[1] = 2;
  } else {              // Rot(a,b,g) = RZ(g) RY(b) RZ(a), Eq. 28
    const M2 za = m_rz(p[0]), yb = m_ry(p[1]), zg = m_rz(p[2]);
    U = mmul(zg, mmul(yb, za));
    Vk[0] = mmul(zg, yb); Gk[0] = 2;
    Vk[1] = zg; Gk[1] = 1;
    Vk[2] = {{1, 0}, {0, 0}, {0, 0}, {1, 0}}; Gk[2] = 2;
  }
  float* g = a.gates + (int64_t)t * 8;
  g[0] = (float)U.a.x; g[1] = (float)U.a.y; g[2] = (float)U.b.x; g[3] = (float)U.b.y;
  g[4] = (float)U.c.x; g[5] = (float)U.c.y; g[6] = (float)U.d.x; g[7] = (float)U.d.y;
  for (int kk = 0; kk < 3; ++kk) {
    float* c = a.cmat + ((int64_t)t * 3 + kk) * 4;
    if (kk < k) pauli_coords(Vk[kk], Gk[kk], c);
    else c[0] = c[1] = c[2] = c[3] = 0.f;
  }
  if (l == 0) pauli_coords(U, a.enc == 0 ? 0 : 1, a.cenc + q * 4);
}

// Diagonal of the CRZ mesh of every layer (Eq. 29): CRZ(c, t)(theta) multiplies |k> by
// exp(i theta (b_t(k) - 1/2)) where b_c(k) = 1, so the whole mesh multiplies |k> by
// exp(i phi_l(k)), phi_l(k) = sum over ordered pairs c != t of theta_ct b_c(k) (b_t(k) - 1/2)
// (b_q(k) = bit n-1-q of k). One thread per (layer, k), FP64; writes (cos, sin) in FP32
// and, if d64 is given, in FP64.
__global__ void crz_phase_kernel(const float* params, int64_t circ_off, int n, int L, int ansatz,
                                 float2* out, double2* d64) {
  const int dim = 1 << n;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)L * dim) return;
  const int l = (int)(i / dim), k = (int)(i % dim);
  const float* th = params + circ_off + (int64_t)l * qp_layer_params(ansatz, n) + n * qp_ansatz_k(ansatz);
  double ph = 0.0;
  for (int c = 0; c < n; ++c) {
    if (!((k >> (n - 1 - c)) & 1)) continue;
    for (int t = 0; t < n; ++t) {
      if (t == c) continue;
      const double bt = ((k >> (n - 1 - t)) & 1) ? 0.5 : -0.5;
      ph += (double)th[c * (n - 1) + (t < c ? t : t - 1)] * bt;
    }
  }
  double sn, cs;
  sincos(ph, &sn, &cs);
  out[i] = make_float2((float)cs, (float)sn);
  if (d64) d64[i] = make_double2(cs, sn);
}

// --------------------------------------------------------------------------- symmetry penalty
// Eq. 18 needs the fields at the mirrored points (-x, y, t) and (x, -y, t) of every collocation
// point; in the dielectric case only (x, -y, t) (the terms mirrored along x are left out).
// Points of set 2 of the main pass: the boundary points, then the mirrored points
// (vacuum: all x-mirrors, then all y-mirrors; dielectric: the y-mirrors).
__global__ void sym_points_kernel(const float* colloc, int64_t nc, const float* bc, int64_t nb, int medium,
                                  float* out) {
  const int64_t nm = medium == 0 ? 2 * nc : nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb + nm; i += (int64_t)gridDim.x * blockDim.x) {
    float x, y, t;
    if (i < nb) {
      x = bc[3 * i]; y = bc[3 * i + 1]; t = bc[3 * i + 2];
    } else {
      const int64_t j = i - nb, p = j % nc;
      const bool mx = medium == 0 && j < nc;
      x = mx ? -colloc[3 * p] : colloc[3 * p];
      y = mx ? colloc[3 * p + 1] : -colloc[3 * p + 1];
      t = colloc[3 * p + 2];
    }
    out[3 * i] = x; out[3 * i + 1] = y; out[3 * i + 2] = t;
  }
}

// From the fields F (global rows: the nc collocation points, then the mirrored points in the
// order above): the per-point sums of Eq. 18 (one FP64 partial per block), the cotangents of
// w_sym L_sym = (w_sym / N) sum_p [...] for the collocation points' fields (gsym) and for the
// mirrored points' fields (gext). 256 threads per block.
__global__ void sym_cot_kernel(const float* F, int64_t nc, int medium, float w_sym, double N, float* gsym,
                               float* gext, double* part) {
  __shared__ double ws[8];
  const float k = (float)(2.0 * w_sym / N);
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nc; p += (int64_t)gridDim.x * blockDim.x) {
    const float* f = F + 3 * p;
    float gc[3] = {0.f, 0.f, 0.f};
    if (medium == 0) {
      const float* m = F + 3 * (nc + p);                 // f(-x, y, t): Ez, Hx even; Hy odd
      const float a = f[0] - m[0], b = f[1] - m[1], c = f[2] + m[2];
      acc += (double)(a * a + b * b + c * c);
      gc[0] += k * a; gc[1] += k * b; gc[2] += k * c;
      float* ge = gext + 3 * p;
      ge[0] = -k * a; ge[1] = -k * b; ge[2] = k * c;
    }
    const int64_t oy = medium == 0 ? nc + p : p;         // row of f(x, -y, t) among the mirrors
    const float* m = F + 3 * (nc + oy);                  // Ez even; Hx odd; Hy even in y
    const float a = f[0] - m[0], b = f[1] + m[1], c = f[2] - m[2];
    acc += (double)(a * a + b * b + c * c);
    gc[0] += k * a; gc[1] += k * b; gc[2] += k * c;
    float* ge = gext + 3 * oy;
    ge[0] = -k * a; ge[1] = k * b; ge[2] = -k * c;
    gsym[3 * p] = gc[0]; gsym[3 * p + 1] = gc[1]; gsym[3 * p + 2] = gc[2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += ws[i];
    part[blockIdx.x] = t;
  }
}

// --------------------------------------------------------------------------- BH indicator
// Sec. 5: U~(t_k) = U(t_k) / U(0) for the energy slices u[0 .. nt), and I_BH = 1 - min over
// the slices k >= k0 (t_k >= delta) of U~(t_k). One warp.
__global__ void bh_indicator_kernel(const double* u, int nt, int k0, double* out) {
  const int lane = threadIdx.x;
  const double u0 = u[0];
  double mn = 1.0 / 0.0;
  for (int k = lane; k < nt; k += 32) {
    const double r = u[k] / u0;
    out[k] = r;
    if (k >= k0) mn = fmin(mn, r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if (lane == 0) out[nt] = 1.0 - mn;
}

// --------------------------------------------------------------------------- premap

struct PremapArgs {
  const float* pts[3];
  int64_t npts[3];
  int64_t ptot;
  const float* params;
  int32_t n, premap, scale, n_direct, F, H;
  float* thetaJ;          // [P][n][4]
  float2* cs;             // [P][n] (cos, sin) of theta / 2 for the tensor-core path, or null
  const float* dthetaJ;   // [P][n][4] (backward)
  float* d1;              // [P][H][4] dL/dh1, dL/dh1_d
  float* d2;              // [P][n][4] dL/dh2, dL/dh2_d
  float* u1;              // [P][H][4] u1, u1_d
  int32_t* counts;
  int32_t medium;
  float disk_r, disk_x0, disk_y0;
  int32_t* status;        // device status word (tensor-core premap: an expired wait), or null
};

// theta = g(h) with a = tanh(h) and one of Eq. 27's scalings; g', g'' in terms of h.
__device__ __forceinline__ void scale_tanh(int s, float h, float& g0, float& g1, float& g2) {
  const float t = tanhf(h);
  const float s2 = 1.f - t * t;
  const float sh = 1.f / coshf(h);
  switch (s) {
    case 0: g0 = t; g1 = s2; g2 = -2.f * t * s2; break;
    case 1: g0 = 3.14159265358979f * t; g1 = 3.14159265358979f * s2; g2 = -2.f * 3.14159265358979f * t * s2; break;
    case 2: g0 = (t + 1.f) * 1.57079632679490f; g1 = 1.57079632679490f * s2; g2 = -3.14159265358979f * t * s2; break;
    case 3: g0 = asinf(t) + 1.57079632679490f; g1 = sh; g2 = -sh * t; break;
    default: g0 = acosf(t); g1 = -sh; g2 = sh * t; break;
  }
}
// Direct premap: theta = scale(v), derivative w.r.t. v.
__device__ __forceinline__ void scale_direct(int s, float v, float& g0, float& g1) {
  switch (s) {
    case 0: g0 = v; g1 = 1.f; break;
    case 1: g0 = 3.14159265358979f * v; g1 = 3.14159265358979f; break;
    case 2: g0 = (v + 1.f) * 1.57079632679490f; g1 = 1.57079632679490f; break;
    case 3: g0 = asinf(v) + 1.57079632679490f; g1 = rsqrtf(fmaxf(1.f - v * v, 1e-30f)); break;
    default: g0 = acosf(v); g1 = -rsqrtf(fmaxf(1.f - v * v, 1e-30f)); break;
  }
}

__device__ __forceinline__ const float* point_ptr(const PremapArgs& a, int64_t gp, int& set, int64_t& li) {
  set = 0;
  li = gp;
  if (li >= a.npts[0]) { li -= a.npts[0]; set = 1; if (li >= a.npts[1]) { li -= a.npts[1]; set = 2; } }
  return a.pts[set] + li * 3;
}

// Hidden layer h1 = W1 r + b1 with r = [cos(Omega v), sin(Omega v)] and its x,y,t tangents.
template <int H>
__device__ __forceinline__ void mlp_hidden(const float* sW1, const float* sb1, const float* om, int F,
                                           float vx, float vy, float vt, float (&h)[H][4]) {
#pragma unroll
  for (int o = 0; o < H; ++o) { h[o][0] = sb1[o]; h[o][1] = h[o][2] = h[o][3] = 0.f; }
  for (int f = 0; f < F; ++f) {
    const float ox = om[3 * f], oy = om[3 * f + 1], ot = om[3 * f + 2];
    float sn, cs;
    sincosf(ox * vx + oy * vy + ot * vt, &sn, &cs);
#pragma unroll
    for (int o = 0; o < H; ++o) {
      const float wc = sW1[o * 2 * F + f], ws = sW1[o * 2 * F + F + f];
      h[o][0] += wc * cs + ws * sn;
      const float q = cs * ws - sn * wc;  // d/du of (wc cos u + ws sin u)
      h[o][1] += q * ox;
      h[o][2] += q * oy;
      h[o][3] += q * ot;
    }
  }
}

template <int H>
__global__ void premap_fwd_kernel(PremapArgs a) {
  extern __shared__ __align__(16) float psm[];
  const int F = a.F, n = a.n;
  float* sW1 = psm;
  float* sb1 = sW1 + H * 2 * F;
  float* sW2 = sb1 + H;
  float* sb2 = sW2 + n * H;
  float* som = sb2 + n;
  if (a.premap == 1) {
    const float* om = a.params;
    const float* W1 = om + 3 * F;
    for (int i = threadIdx.x; i < 3 * F; i += blockDim.x) som[i] = om[i];
    for (int i = threadIdx.x; i < H * 2 * F; i += blockDim.x) sW1[i] = W1[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) sb1[i] = W1[H * 2 * F + i];
    for (int i = threadIdx.x; i < n * H; i += blockDim.x) sW2[i] = W1[H * 2 * F + H + i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) sb2[i] = W1[H * 2 * F + H + n * H + i];
    __syncthreads();
  }
  for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < a.ptot;
       gp += (int64_t)gridDim.x * blockDim.x) {
    int set;
    int64_t li;
    const float* v = point_ptr(a, gp, set, li);
    const float vx = v[0], vy = v[1], vt = v[2];
    float4* out = reinterpret_cast<float4*>(a.thetaJ) + gp * n;
    if (a.medium == 1 && set == 0) {
      const float dx = vx - a.disk_x0, dy = vy - a.disk_y0;
      if (__fmaf_rn(dx, dx, dy * dy) < a.disk_r * a.disk_r) atomicAdd(&a.counts[0], 1);
    }
    if (a.premap == 0) {
      const float vv[3] = {vx, vy, vt};
      for (int q = 0; q < n; ++q) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < a.n_direct) {
          float g0, g1;
          scale_direct(a.scale, vv[q], g0, g1);
          o.x = g0;
          if (q == 0) o.y = g1;
          if (q == 1) o.z = g1;
          if (q == 2) o.w = g1;
        }
        out[q] = o;
      }
      continue;
    }
    float h[H][4];
    mlp_hidden<H>(sW1, sb1, som, F, vx, vy, vt, h);
#pragma unroll
    for (int o = 0; o < H; ++o) {
      const float u = tanhf(h[o][0]);
      const float du = 1.f - u * u;
      h[o][0] = u;
      h[o][1] *= du; h[o][2] *= du; h[o][3] *= du;
    }
    for (int j = 0; j < n; ++j) {
      float z0 = sb2[j], z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
      for (int o = 0; o < H; ++o) {
        const float w = sW2[j * H + o];
        z0 += w * h[o][0]; z1 += w * h[o][1]; z2 += w * h[o][2]; z3 += w * h[o][3];
      }
      float g0, g1, g2;
      scale_tanh(a.scale, z0, g0, g1, g2);
      out[j] = make_float4(g0, g1 * z1, g1 * z2, g1 * z3);
    }
  }
}

// ---- RFF + MLP premap, four threads per point (each owns H/4 hidden units)
// The block's 32 points get their [cos, sin](Omega v) table once in shared memory; the first
// layer's weights are kept transposed ([2F][H]) so a thread reads its H/4 units contiguously;
// the output layer is summed over the four lanes of a point with two butterfly shuffles.
__host__ __device__ inline int premap4_smem(int F, int H, int n) {
  const int wfl = 2 * F * H + H + n * H + n + 3 * F;
  return ((wfl + 3) & ~3) * 4 + 32 * (F + 1) * 8;
}

struct Premap4Smem {
  float *w1t, *b1, *w2, *b2, *om;
  float2* sc;
};
__device__ __forceinline__ Premap4Smem premap4_load(const PremapArgs& a, float* psm) {
  const int F = a.F, n = a.n, H = a.H;
  Premap4Smem m;
  m.w1t = psm;
  m.b1 = m.w1t + 2 * F * H;
  m.w2 = m.b1 + H;
  m.b2 = m.w2 + n * H;
  m.om = m.b2 + n;
  m.sc = reinterpret_cast<float2*>(psm + ((2 * F * H + H + n * H + n + 3 * F + 3) & ~3));
  const float* om = a.params;
  const float* W1 = om + 3 * F;
  for (int i = threadIdx.x; i < 3 * F; i += blockDim.x) m.om[i] = om[i];
  for (int i = threadIdx.x; i < H * 2 * F; i += blockDim.x) {
    const int o = i / (2 * F), k = i % (2 * F);
    m.w1t[k * H + o] = W1[i];
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) m.b1[i] = W1[H * 2 * F + i];
  for (int i = threadIdx.x; i < n * H; i += blockDim.x) m.w2[i] = W1[H * 2 * F + H + i];
  for (int i = threadIdx.x; i < n; i += blockDim.x) m.b2[i] = W1[H * 2 * F + H + n * H + i];
  return m;
}

// [cos, sin](Omega v) of the block's 32 points starting at p0 (rows of F + 1 entries).
__device__ __forceinline__ void premap4_table(const PremapArgs& a, const Premap4Smem& m, int64_t p0) {
  const int F = a.F;
  for (int e = threadIdx.x; e < 32 * F; e += blockDim.x) {
    const int pi = e / F, f = e % F;
    const int64_t gp = p0 + pi;
    float2 v = make_float2(1.f, 0.f);
    if (gp < a.ptot) {
      int set;
      int64_t li;
      const float* x = point_ptr(a, gp, set, li);
      float sn, cs;
      sincosf(m.om[3 * f] * x[0] + m.om[3 * f + 1] * x[1] + m.om[3 * f + 2] * x[2], &sn, &cs);
      v = make_float2(cs, sn);
    }
    m.sc[pi * (F + 1) + f] = v;
  }
}

// Hidden layer of this thread's units (pre-activation and x, y, t tangents).
template <int QH>
__device__ __forceinline__ void premap4_hidden(const PremapArgs& a, const Premap4Smem& m, int pl, int ob,
                                               float (&h)[QH][4]) {
  const int F = a.F, H = a.H;
#pragma unroll
  for (int k = 0; k < QH; ++k) { h[k][0] = m.b1[ob + k]; h[k][1] = h[k][2] = h[k][3] = 0.f; }
  for (int f = 0; f < F; ++f) {
    const float2 c = m.sc[pl * (F + 1) + f];
    const float ox = m.om[3 * f], oy = m.om[3 * f + 1], ot = m.om[3 * f + 2];
    const float* wc = m.w1t + f * H + ob;
    const float* wsn = m.w1t + (F + f) * H + ob;
#pragma unroll
    for (int k = 0; k < QH; ++k) {
      h[k][0] += wc[k] * c.x + wsn[k] * c.y;
      const float q = c.x * wsn[k] - c.y * wc[k];  // d/du of (wc cos u + ws sin u)
      h[k][1] += q * ox;
      h[k][2] += q * oy;
      h[k][3] += q * ot;
    }
  }
}

// Sum of a value over the four lanes of a point.
__device__ __forceinline__ float quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

template <int H>
__global__ void __launch_bounds__(128) premap_fwd4_kernel(PremapArgs a) {
  constexpr int QH = H / 4;
  extern __shared__ __align__(16) float psm[];
  const Premap4Smem m = premap4_load(a, psm);
  const int n = a.n;
  const int pl = threadIdx.x >> 2, oq = threadIdx.x & 3, ob = oq * QH;
  for (int64_t p0 = blockIdx.x * 32LL; p0 < a.ptot; p0 += gridDim.x * 32LL) {
    __syncthreads();  // weights loaded / the previous points' table consumed
    premap4_table(a, m, p0);
    __syncthreads();
    const int64_t gp = p0 + pl;
    const bool act = gp < a.ptot;
    float h[QH][4];
    premap4_hidden<QH>(a, m, pl, ob, h);
#pragma unroll
    for (int k = 0; k < QH; ++k) {
      const float u = tanhf(h[k][0]);
      const float du = 1.f - u * u;
      h[k][0] = u;
      h[k][1] *= du; h[k][2] *= du; h[k][3] *= du;
    }
    float4* out = reinterpret_cast<float4*>(a.thetaJ) + gp * n;
    for (int j = 0; j < n; ++j) {
      float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
      for (int k = 0; k < QH; ++k) {
        const float w = m.w2[j * H + ob + k];
        z0 += w * h[k][0]; z1 += w * h[k][1]; z2 += w * h[k][2]; z3 += w * h[k][3];
      }
      z0 = quad_sum(z0) + m.b2[j];
      z1 = quad_sum(z1); z2 = quad_sum(z2); z3 = quad_sum(z3);
      if (act && oq == (j & 3)) {
        float g0, g1, g2;
        scale_tanh(a.scale, z0, g0, g1, g2);
        out[j] = make_float4(g0, g1 * z1, g1 * z2, g1 * z3);
      }
    }
    if (act && oq == 0 && a.medium == 1) {
      int set;
      int64_t li;
      const float* v = point_ptr(a, gp, set, li);
      if (set == 0) {
        const float dx = v[0] - a.disk_x0, dy = v[1] - a.disk_y0;
        if (__fmaf_rn(dx, dx, dy * dy) < a.disk_r * a.disk_r) atomicAdd(&a.counts[0], 1);
      }
    }
  }
}

// Backward of the premap with four threads per point (see premap_bwd_kernel for the algebra).
template <int H>
__global__ void __launch_bounds__(128) premap_bwd4_kernel(PremapArgs a) {
  constexpr int QH = H / 4;
  extern __shared__ __align__(16) float psm[];
  const Premap4Smem m = premap4_load(a, psm);
  const int n = a.n;
  const int pl = threadIdx.x >> 2, oq = threadIdx.x & 3, ob = oq * QH;
  for (int64_t p0 = blockIdx.x * 32LL; p0 < a.ptot; p0 += gridDim.x * 32LL) {
    __syncthreads();
    premap4_table(a, m, p0);
    __syncthreads();
    const int64_t gp = p0 + pl;
    const bool act = gp < a.ptot;
    const int64_t gpc = act ? gp : 0;
    float h[QH][4], hd[QH][4];
    premap4_hidden<QH>(a, m, pl, ob, h);
#pragma unroll
    for (int k = 0; k < QH; ++k) {
      const float u = tanhf(h[k][0]);
      const float du = 1.f - u * u;
      hd[k][0] = u;
      hd[k][1] = h[k][1]; hd[k][2] = h[k][2]; hd[k][3] = h[k][3];
      h[k][0] = u;
      h[k][1] *= du; h[k][2] *= du; h[k][3] *= du;
    }
    if (act) {
      float4* u1o = reinterpret_cast<float4*>(a.u1) + gp * H + ob;
#pragma unroll
      for (int k = 0; k < QH; ++k) u1o[k] = make_float4(h[k][0], h[k][1], h[k][2], h[k][3]);
    }
    float gu[QH][4];
#pragma unroll
    for (int k = 0; k < QH; ++k) gu[k][0] = gu[k][1] = gu[k][2] = gu[k][3] = 0.f;
    const float4* dtj = reinterpret_cast<const float4*>(a.dthetaJ) + gpc * n;
    float4* d2o = reinterpret_cast<float4*>(a.d2) + gpc * n;
    for (int j = 0; j < n; ++j) {
      float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
      for (int k = 0; k < QH; ++k) {
        const float w = m.w2[j * H + ob + k];
        z0 += w * h[k][0]; z1 += w * h[k][1]; z2 += w * h[k][2]; z3 += w * h[k][3];
      }
      z0 = quad_sum(z0) + m.b2[j];
      z1 = quad_sum(z1); z2 = quad_sum(z2); z3 = quad_sum(z3);
      float g0, g1, g2;
      scale_tanh(a.scale, z0, g0, g1, g2);
      const float4 dt = dtj[j];
      // theta = g(z0), J_d = g'(z0) z_d
      const float dz1 = dt.y * g1, dz2 = dt.z * g1, dz3 = dt.w * g1;
      const float dz0 = dt.x * g1 + g2 * (dt.y * z1 + dt.z * z2 + dt.w * z3);
      if (act && oq == (j & 3)) d2o[j] = make_float4(dz0, dz1, dz2, dz3);
#pragma unroll
      for (int k = 0; k < QH; ++k) {
        const float w = m.w2[j * H + ob + k];
        gu[k][0] += w * dz0; gu[k][1] += w * dz1; gu[k][2] += w * dz2; gu[k][3] += w * dz3;
      }
    }
    if (act) {
      float4* d1o = reinterpret_cast<float4*>(a.d1) + gp * H + ob;
#pragma unroll
      for (int k = 0; k < QH; ++k) {
        const float u = hd[k][0];
        const float du = 1.f - u * u;
        // u1_d = du * h1_d; d du / d h1 = -2 u du
        const float g1x = gu[k][1] * du, g1y = gu[k][2] * du, g1t = gu[k][3] * du;
        const float g10 = gu[k][0] * du -
                          2.f * u * du * (gu[k][1] * hd[k][1] + gu[k][2] * hd[k][2] + gu[k][3] * hd[k][3]);
        d1o[k] = make_float4(g10, g1x, g1y, g1t);
      }
    }
  }
}

// Per-point backward through scale, output layer and tanh hidden layer, given
// dL/dtheta_j and dL/dJ_jd from the circuit's adjoint sweep.
template <int H>
__global__ void premap_bwd_kernel(PremapArgs a) {
  extern __shared__ __align__(16) float psm[];
  const int F = a.F, n = a.n;
  float* sW1 = psm;
  float* sb1 = sW1 + H * 2 * F;
  float* sW2 = sb1 + H;
  float* sb2 = sW2 + n * H;
  float* som = sb2 + n;
  {
    const float* om = a.params;
    const float* W1 = om + 3 * F;
    for (int i = threadIdx.x; i < 3 * F; i += blockDim.x) som[i] = om[i];
    for (int i = threadIdx.x; i < H * 2 * F; i += blockDim.x) sW1[i] = W1[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) sb1[i] = W1[H * 2 * F + i];
    for (int i = threadIdx.x; i < n * H; i += blockDim.x) sW2[i] = W1[H * 2 * F + H + i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) sb2[i] = W1[H * 2 * F + H + n * H + i];
    __syncthreads();
  }
  for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < a.ptot;
       gp += (int64_t)gridDim.x * blockDim.x) {
    int set;
    int64_t li;
    const float* v = point_ptr(a, gp, set, li);
    float h[H][4];
    mlp_hidden<H>(sW1, sb1, som, F, v[0], v[1], v[2], h);
    float hd[H][4];  // tangents of h1 kept for the second-order term
#pragma unroll
    for (int o = 0; o < H; ++o) {
      const float u = tanhf(h[o][0]);
      const float du = 1.f - u * u;
      hd[o][0] = u;
      hd[o][1] = h[o][1]; hd[o][2] = h[o][2]; hd[o][3] = h[o][3];
      h[o][0] = u;
      h[o][1] *= du; h[o][2] *= du; h[o][3] *= du;
    }
    float4* u1o = reinterpret_cast<float4*>(a.u1) + gp * H;
#pragma unroll
    for (int o = 0; o < H; ++o) u1o[o] = make_float4(h[o][0], h[o][1], h[o][2], h[o][3]);
    // dL/du1 and dL/du1_d accumulated over outputs j
    float gu[H][4];
#pragma unroll
    for (int o = 0; o < H; ++o) gu[o][0] = gu[o][1] = gu[o][2] = gu[o][3] = 0.f;
    const float4* dtj = reinterpret_cast<const float4*>(a.dthetaJ) + gp * n;
    float4* d2o = reinterpret_cast<float4*>(a.d2) + gp * n;
    for (int j = 0; j < n; ++j) {
      float z0 = sb2[j], z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
      for (int o = 0; o < H; ++o) {
        const float w = sW2[j * H + o];
        z0 += w * h[o][0]; z1 += w * h[o][1]; z2 += w * h[o][2]; z3 += w * h[o][3];
      }
      float g0, g1, g2;
      scale_tanh(a.scale, z0, g0, g1, g2);
      const float4 dt = dtj[j];
      // theta = g(z0), J_d = g'(z0) z_d
      const float dz1 = dt.y * g1, dz2 = dt.z * g1, dz3 = dt.w * g1;
      const float dz0 = dt.x * g1 + g2 * (dt.y * z1 + dt.z * z2 + dt.w * z3);
      d2o[j] = make_float4(dz0, dz1, dz2, dz3);
#pragma unroll
      for (int o = 0; o < H; ++o) {
        const float w = sW2[j * H + o];
        gu[o][0] += w * dz0; gu[o][1] += w * dz1; gu[o][2] += w * dz2; gu[o][3] += w * dz3;
      }
    }
    float4* d1o = reinterpret_cast<float4*>(a.d1) + gp * H;
#pragma unroll
    for (int o = 0; o < H; ++o) {
      const float u = hd[o][0];
      const float du = 1.f - u * u;
      // u1_d = du * h1_d; d du / d h1 = -2 u du
      const float g1x = gu[o][1] * du, g1y = gu[o][2] * du, g1t = gu[o][3] * du;
      const float g10 = gu[o][0] * du -
                        2.f * u * du * (gu[o][1] * hd[o][1] + gu[o][2] * hd[o][2] + gu[o][3] * hd[o][3]);
      d1o[o] = make_float4(g10, g1x, g1y, g1t);
    }
  }
}

// ---- RFF + MLP premap with F = 64, H = 32: shared constants and the tile loader of the
// tensor-core kernels (qp_premap_tc.cuh).
// With r = [cos(Omega v), sin(Omega v)] (K = 2F = 128 features), unit o's pre-activation and
// its x, y, t tangents are h_c[o] = sum_i B[(o, c)][i] r[i] with
//   B[(o, 0)][i] = W1[o][i],  B[(o, c)][f] = W1[o][F + f] Omega[f][c],  B[(o, c)][F + f] = -W1[o][f] Omega[f][c]
// (d/dv_c turns cos into -sin Omega and sin into cos Omega: the halves swap), so the forward is
// one GEMM [points] x [K] x [N = 4H = 128 columns (o, c)] and needs no tangent rows. The weight
// gradient is the transposed contraction over points, D[(o, c)][i] = sum_p d1_p[(o, c)] r_p[i],
// folded back by the same rule:
//   dW1[o][f] = D[(o,0)][f] - sum_c Omega[f][c] D[(o,c)][F+f],  dW1[o][F+f] = D[(o,0)][F+f] + sum_c Omega[f][c] D[(o,c)][f].
// The forward keeps u = tanh(h_0) and its tangents u_c = (1 - u^2) h_c per point for the
// backward (the backward needs no h_c: (1 - u^2) h_c = u_c).
constexpr int PG_F = 64, PG_H = 32, PG_K = 2 * PG_F, PG_N = 4 * PG_H, PG_TP = 64, PG_THREADS = 256;
constexpr int PG_US = PG_H + 1;   // padded row of the per-point unit table (float4)
// the tile's point coordinates
__device__ __forceinline__ void pg_load_points(const PremapArgs& a, int64_t p0, float* Ps) {
  for (int e = threadIdx.x; e < PG_TP * 3; e += blockDim.x) {
    const int64_t gp = p0 + e / 3;
    float v = 0.f;
    if (gp < a.ptot) {
      int set;
      int64_t li;
      v = point_ptr(a, gp, set, li)[e % 3];
    }
    Ps[e] = v;
  }
}


// Weight gradients of the premap as block partials over contiguous point chunks.
//   dW1[o][i] = sum_p d1[o].(r_i, r_{i,x}, r_{i,y}, r_{i,t}),  db1[o] = sum_p d1[o].x
//   dW2[j][o] = sum_p d2[j].(u1[o] with tangents),             db2[j] = sum_p d2[j].x
struct WgradArgs {
  PremapArgs p;
  float* part;        // [grid][nW]
  int32_t nW;         // H*2F + H + n*H + n
  int32_t tile;       // points per shared-memory tile
};

__global__ void premap_wgrad_kernel(WgradArgs w) {
  extern __shared__ __align__(16) float wsm[];
  const PremapArgs& a = w.p;
  const int F = a.F, n = a.n, H = a.H, TP = w.tile;
  const int F2 = 2 * F;
  float4* rt = reinterpret_cast<float4*>(wsm);          // [TP][2F]
  float4* dt = rt + TP * F2;                            // [TP][H]
  float4* ut = dt + TP * H;                             // [TP][H]
  float4* d2t = ut + TP * H;                            // [TP][n]
  float* om = reinterpret_cast<float*>(d2t + TP * n);   // [F][3]
  for (int i = threadIdx.x; i < 3 * F; i += blockDim.x) om[i] = a.params[i];
  const int nb1 = (H / 4) * (F2 / 4);   // 4x4 blocks of dW1
  const int nth = blockDim.x;
  // per-thread accumulators: up to WS blocks of dW1 (16 each), WS dW2 entries, WS biases
  constexpr int WS = 4;
  float acc1[WS][16];
  float acc2[WS], accb[WS];
#pragma unroll
  for (int s = 0; s < WS; ++s) {
    acc2[s] = 0.f; accb[s] = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) acc1[s][k] = 0.f;
  }
  const int64_t chunk = (a.ptot + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = blockIdx.x * chunk;
  const int64_t p1 = p0 + chunk < a.ptot ? p0 + chunk : a.ptot;
  __syncthreads();
  for (int64_t tb = p0; tb < p1; tb += TP) {
    const int cnt = (int)((p1 - tb) < TP ? (p1 - tb) : TP);
    // stage r (with tangents), d1, u1, d2 of the tile
    for (int e = threadIdx.x; e < cnt * F; e += nth) {
      const int pi = e / F, f = e % F;
      int set;
      int64_t li;
      const float* v = point_ptr(a, tb + pi, set, li);
      const float ox = om[3 * f], oy = om[3 * f + 1], ot = om[3 * f + 2];
      float sn, cs;
      sincosf(ox * v[0] + oy * v[1] + ot * v[2], &sn, &cs);
      rt[pi * F2 + f] = make_float4(cs, -sn * ox, -sn * oy, -sn * ot);
      rt[pi * F2 + F + f] = make_float4(sn, cs * ox, cs * oy, cs * ot);
    }
    for (int e = threadIdx.x; e < cnt * H; e += nth) {
      dt[e] = reinterpret_cast<const float4*>(a.d1)[tb * H + e];
      ut[e] = reinterpret_cast<const float4*>(a.u1)[tb * H + e];
    }
    for (int e = threadIdx.x; e < cnt * n; e += nth) d2t[e] = reinterpret_cast<const float4*>(a.d2)[tb * n + e];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < WS; ++s) {
      const int blk = threadIdx.x + s * nth;
      if (blk < nb1) {
        const int ob = blk / (F2 / 4), ib = blk % (F2 / 4);
        for (int pi = 0; pi < cnt; ++pi) {
          float4 d[4], r[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) { d[k] = dt[pi * H + ob * 4 + k]; r[k] = rt[pi * F2 + ib * 4 + k]; }
#pragma unroll
          for (int oo = 0; oo < 4; ++oo)
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
              acc1[s][oo * 4 + ii] += d[oo].x * r[ii].x + d[oo].y * r[ii].y + d[oo].z * r[ii].z + d[oo].w * r[ii].w;
        }
      }
      const int e2 = threadIdx.x + s * nth;
      if (e2 < n * H) {
        const int j = e2 / H, o = e2 % H;
        for (int pi = 0; pi < cnt; ++pi) {
          const float4 d = d2t[pi * n + j], u = ut[pi * H + o];
          acc2[s] += d.x * u.x + d.y * u.y + d.z * u.z + d.w * u.w;
        }
      }
      const int eb = threadIdx.x + s * nth;
      if (eb < H + n) {
        for (int pi = 0; pi < cnt; ++pi) accb[s] += eb < H ? dt[pi * H + eb].x : d2t[pi * n + eb - H].x;
      }
    }
    __syncthreads();
  }
  float* out = w.part + (int64_t)blockIdx.x * w.nW;
  // partial layout: [dW1 (H x 2F)][db1 (H)][dW2 (n x H)][db2 (n)] == parameter layout order
#pragma unroll
  for (int s = 0; s < WS; ++s) {
    const int blk = threadIdx.x + s * nth;
    if (blk < nb1) {
      const int ob = blk / (F2 / 4), ib = blk % (F2 / 4);
#pragma unroll
      for (int oo = 0; oo < 4; ++oo)
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) out[(ob * 4 + oo) * F2 + ib * 4 + ii] = acc1[s][oo * 4 + ii];
    }
    const int e2 = threadIdx.x + s * nth;
    if (e2 < n * H) out[H * F2 + H + e2] = acc2[s];
    const int eb = threadIdx.x + s * nth;
    if (eb < H + n) out[eb < H ? H * F2 + eb : H * F2 + H + n * H + (eb - H)] = accb[s];
  }
}

// Number of points strictly inside the dielectric disk (the same float32 test as the loss).
__global__ void count_dielectric_kernel(const float* pts, int64_t n, float x0, float y0, float r,
                                        unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float dx = pts[3 * i] - x0, dy = pts[3 * i + 1] - y0;
    c += __fmaf_rn(dx, dx, dy * dy) < r * r ? 1ull : 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// --------------------------------------------------------------------------- final reduce

struct ReduceArgs {
  const double* blk_loss;
  const float* blk_grad;
  int32_t nblk, loss_stride, grad_stride;
  const float* wpart;
  int32_t nwblk, nW;
  const float* cmat;
  const int32_t* counts;
  int32_t* status;
  double* loss;
  float* grad;
  int64_t nparams, circ_off, head_off, mlp_off, mlp_count;
  int32_t n, L, m, k, nt, medium, ansatz, phys_loss;
  int32_t nE;                  // gate-gradient partial sums per block (head partials follow)
  const double* sym_part;      // symmetry penalty: per-block sums of Eq. 18, or null
  int32_t nsym;
  float w_sym;
  int64_t nc, ni, nb;          // mean denominators of the three sets
  int64_t norm_diel;           // whole-set points inside the disk, or -1: the counted ones
  float w_ic, w_bc, w_energy;
  int32_t nmain_blocks;        // blocks of the one-warp-per-output part
  int32_t mlp_blocks;          // blocks after them for the premap weights (0: warps per output)
};

// Compensated FP32 sum (Neumaier's variant of Kahan summation): s + c carries the sum of the
// added values to about twice FP32 precision, on the FP32 pipes.
struct CSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ void add(const CSum& o) { add(o.s); c += o.c; }
  __device__ __forceinline__ float value() const { return s + c; }
  __device__ __forceinline__ double dvalue() const { return (double)s + (double)c; }
};

// One warp per output: parameter gradients (the lanes split the block partials), then the
// loss terms and the energy slices; the premap weights in blocks of 32 consecutive outputs
// after them (8 warps split the partial slots, each warp load one contiguous 128-byte row
// piece). The FP32 gradient partials are summed per lane in compensated FP32 (B300's FP64
// pipe is a small fraction of its FP32 rate), then across lanes in FP64; the FP64 loss and
// energy partials in FP64.
__device__ __forceinline__ double warp_sum_dbl(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__global__ void reduce_kernel(ReduceArgs a) {
  const int lane = threadIdx.x & 31;
  if ((int)blockIdx.x >= a.nmain_blocks) {
    // (the whole block takes this branch)
    __shared__ double mpart[8][32];
    const int w = threadIdx.x >> 5;
    const int64_t wi = (int64_t)(blockIdx.x - a.nmain_blocks) * 32 + lane;
    CSum t;
    if (wi < a.mlp_count)
      for (int b = w; b < a.nwblk; b += 8) t.add(a.wpart[(int64_t)b * a.nW + wi]);
    mpart[w][lane] = t.dvalue();
    __syncthreads();
    if (w == 0 && wi < a.mlp_count) {
      double sum = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) sum += mpart[k][lane];
      a.grad[a.mlp_off + wi] = (float)sum;
    }
    return;
  }
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (gw < a.nparams) {
    const int64_t i = gw;
    float val = 0.f;
    if (i >= a.circ_off && i < a.head_off) {
      const int64_t r = i - a.circ_off;
      const int per = qp_layer_params(a.ansatz, a.n);
      const int l = (int)(r / per), w = (int)(r % per);
      if (w < a.n * a.k) {
        // single-qubit angle: Pauli contractions of its gate combined by the coordinates
        const int64_t lq = (int64_t)l * a.n + w / a.k;
        const int kk = w % a.k;
        const float* c = a.cmat + (lq * 3 + kk) * 4;
        CSum s0, s1, s2;
        for (int b = lane; b < a.nblk; b += 32) {
          const float* g = a.blk_grad + (int64_t)b * a.grad_stride + lq * 3;
          s0.add(g[0]); s1.add(g[1]); s2.add(g[2]);
        }
        const double e0 = warp_sum_dbl(s0.dvalue()), e1 = warp_sum_dbl(s1.dvalue()), e2 = warp_sum_dbl(s2.dvalue());
        val = (float)(c[0] * e0 + c[1] * e1 + c[2] * e2);
      } else {
        // CRZ(c, t) angle: generator |1><1|_c (x) Z_t = (Z_t - Z_c Z_t) / 2, so the gradient
        // is (Z_t - Z_ct) / 2 from the layer's Z-correlation sums
        const int pi = w - a.n * a.k, c = pi / (a.n - 1), tj = pi % (a.n - 1);
        const int t = tj < c ? tj : tj + 1;
        const int64_t base = 3LL * a.n * a.L + (int64_t)l * qp_crz_sums(a.ansatz, a.n);
        const int64_t ot = base + t;
        const int64_t oct = base + a.n + qp_pair_index(a.n, c < t ? c : t, c < t ? t : c);
        CSum st, sct;
        for (int b = lane; b < a.nblk; b += 32) {
          st.add(a.blk_grad[(int64_t)b * a.grad_stride + ot]);
          sct.add(a.blk_grad[(int64_t)b * a.grad_stride + oct]);
        }
        const double zt = warp_sum_dbl(st.dvalue()), zct = warp_sum_dbl(sct.dvalue());
        val = (float)(0.5 * (zt - zct));
      }
    } else if (i >= a.head_off) {
      const int64_t hi = a.nE + (i - a.head_off);
      CSum t;
      for (int b = lane; b < a.nblk; b += 32) t.add(a.blk_grad[(int64_t)b * a.grad_stride + hi]);
      val = (float)warp_sum_dbl(t.dvalue());
    } else if (i >= a.mlp_off && a.mlp_count > 0) {
      if (a.mlp_blocks > 0) return;   // written by the premap-weight blocks
      const int64_t wi = i - a.mlp_off;
      CSum t;
      for (int b = lane; b < a.nwblk; b += 32) t.add(a.wpart[(int64_t)b * a.nW + wi]);
      val = (float)warp_sum_dbl(t.dvalue());
    }
    if (lane == 0) a.grad[i] = val;
  } else if (gw == a.nparams) {
    double s[QP_NLP];
#pragma unroll
    for (int k = 0; k < QP_NLP; ++k) s[k] = 0.0;
    for (int b = lane; b < a.nblk; b += 32)
#pragma unroll
      for (int k = 0; k < QP_NLP; ++k) s[k] += a.blk_loss[(int64_t)b * a.loss_stride + k];
#pragma unroll
    for (int k = 0; k < QP_NLP; ++k) s[k] = warp_sum_dbl(s[k]);
    if (lane == 0) {
      const double N = (double)a.nc;
      const double nd = a.medium == 1 ? (a.norm_diel >= 0 ? (double)a.norm_diel : (double)a.counts[0]) : 0.0;
      const double nv = N - nd;
      double m1v = 0, m1d = 0;
      if (a.medium == 1 && a.phys_loss == 1) {
        if (N > 0) m1v = s[0] / N;   // Eq. 35: one MSE over all collocation points
      } else if (a.medium == 1) {
        if (nv > 0) m1v = s[0] / nv;
        if (nd > 0) m1d = s[1] / nd;
      } else if (N > 0) {
        m1v = s[0] / N;
      }
      const double m2 = N > 0 ? s[2] / N : 0, m3 = N > 0 ? s[3] / N : 0;
      const double phys = m1v + m1d + m2 + m3;
      const double en = N > 0 ? a.w_energy * s[4] / N : 0;
      const double ic = a.ni > 0 ? a.w_ic * s[5] / (double)a.ni : 0;
      const double bc = a.nb > 0 ? a.w_bc * s[6] / (double)a.nb : 0;
      double sym = 0.0;
      if (a.w_sym > 0.f) {
        if (a.sym_part && N > 0) {
          for (int b = 0; b < a.nsym; ++b) sym += a.sym_part[b];
          sym *= (double)a.w_sym / N;
        }
        a.loss[QP_NLOSS_OUT + a.nt] = sym;   // w_sym L_sym after the energy slices
      }
      const double tot = phys + ic + bc + en + sym;
      a.loss[0] = tot; a.loss[1] = phys; a.loss[2] = ic; a.loss[3] = bc; a.loss[4] = en;
      a.loss[5] = m1v; a.loss[6] = m1d; a.loss[7] = m2; a.loss[8] = m3;
      if (!isfinite(tot)) atomicCAS(a.status, 0, (int)5);   // an earlier error code stands
    }
  } else if (gw <= a.nparams + a.nt) {
    const int64_t i = gw - a.nparams - 1;
    double u = 0;
    for (int b = lane; b < a.nblk; b += 32) u += a.blk_loss[(int64_t)b * a.loss_stride + QP_NLP + i];
    u = warp_sum_dbl(u);
    if (lane == 0) a.loss[QP_NLOSS_OUT + i] = u;
  }
}

}  // namespace qpk
