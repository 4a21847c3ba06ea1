// qp_mlp.cuh -- the RFF + tanh MLP premap of any depth and width (Sec. 2.2 architecture: RFF
// features, fully connected tanh layers, a linear layer to one angle per qubit, Eq. 27
// scaling), forward with its input tangents and backward with the weight gradients.
//
// Every point carries four rows through the network: the value and its derivatives along x, y
// and t (forward-mode tangents); row (p, s) is s = 0 the value, s = 1..3 the x, y, t tangent.
// For a tanh layer with pre-activation h = W u + b the rows are
//   y0 = tanh(h0),  y_d = s z_d  with  s = 1 - y0^2,  z_d = W u_d  (the pre-tangents),
// and the layer stores its outputs (y0, y_x, y_y, y_t), the next layer's input rows as they
// stand. Its backward, from the cotangents dU of (y0, y_d), is
//   dH0 = s dU0 - 2 y0 sum_d y_d dU_d,   dZ_d = s dU_d,
//   dW += dH0 u0^T + sum_d dZ_d u_d^T,  db += dH0,   dU_prev = W^T (dH0 | dZ_d).
// The first layer's input is r = [cos(Omega v), sin(Omega v)] with tangents
// [-sin(Omega v) Omega_d, cos(Omega v) Omega_d]. The output layer gives theta = g(h),
// J_d = g'(h) h_d (Eq. 27 on a = tanh(h)); its backward is
//   dH = g'(h) dtheta + g''(h) sum_d h_d dJ_d,   dH_d = g'(h) dJ_d.
//
// The layers' contractions over all rows (C = X W^T forward, dU = cot W and dW = cot^T X
// backward) are plain GEMMs, run by the host as library calls on the tensor cores; the kernels
// here are the point-coupled parts around them (features, tanh and its derivative, the output
// scaling, bias and period gradients). Every row buffer and weight copy has its width rounded
// up to four floats (16-byte aligned rows, so that the library takes its vectorised tensor-core
// kernels) with zero pad columns, so the GEMMs run on the padded sizes.
#pragma once
#include <cuda_runtime.h>

#include "qp_common.h"
#include "qp_aux.cuh"

namespace qpm {

struct MlpArgs {
  // points of the call (three sets in order), global point index gp = set base + local index
  const float* pts[3];
  int64_t npts[3];
  int64_t ptot;
  const float* omega;       // [F][3], or [F][6] with the periodic map (fixed RFF frequencies)
  int32_t F;
  const float* period;      // periodic input map (Eqs. 25-26): the learned time period T, or null
  // the layer: out x in weights (row-major [out][in]) and bias; row strides of its input and
  // output row buffers
  const float* W;
  const float* b;
  int32_t in, out, ldi, ldo;
  const float* act_in;      // previous layer's outputs, rows by mlp_row (null for the first layer)
  float* act_out;           // hidden layer: its outputs, rows by mlp_row
  int64_t n4;               // the first n4 points carry four rows (value and x, y, t tangents),
                            // the others one (no later stage reads their input derivatives)
  // output layer
  int32_t scale;            // Eq. 27 scaling
  float* thetaJ;            // [P][out] float4 (theta, J_x, J_y, J_t)
  float* hout;              // [P][out] float4 (h, h_x, h_y, h_t)
  // dielectric-set count of the loss (output layer of the forward)
  int32_t* counts;
  int32_t medium;
  float disk_r, disk_x0, disk_y0;
};

// First row of point gp in a row buffer: four rows for each of the first n4 points, then one.
__host__ __device__ __forceinline__ int64_t mlp_row(int64_t gp, int64_t n4) { return gp < n4 ? 4 * gp : 3 * n4 + gp; }

__device__ __forceinline__ const float* mlp_point(const MlpArgs& a, int64_t gp, int& set) {
  set = 0;
  int64_t li = gp;
  if (li >= a.npts[0]) { li -= a.npts[0]; set = 1; if (li >= a.npts[1]) { li -= a.npts[1]; set = 2; } }
  return a.pts[set] + li * 3;
}

// Input map of point v, computed once per point: u = v, or with the periodic map (Eqs. 25-26)
// u = (sin pi x, cos pi x, sin pi y, cos pi y, sin phi, cos phi) with phi = w t, w = 2 pi / T.
struct RffMap {
  float u[6];
  float w, t;
  float dphi, wT;   // periodic map: d phi / dT = -phi / T and w / T
};
__device__ __forceinline__ RffMap rff_map(const MlpArgs& a, const float* v) {
  RffMap m;
  m.t = v[2];
  if (!a.period) {
    m.u[0] = v[0]; m.u[1] = v[1]; m.u[2] = v[2];
    m.u[3] = m.u[4] = m.u[5] = 0.f;
    m.w = m.dphi = m.wT = 0.f;
    return m;
  }
  const float T = __ldg(a.period);
  m.w = 6.28318530717959f / T;
  m.dphi = -(m.w * v[2]) / T;
  m.wT = m.w / T;
  float sx, cx, sy, cy, st, ct;
  sincospif(v[0], &sx, &cx);
  sincospif(v[1], &sy, &cy);
  sincosf(m.w * v[2], &st, &ct);
  m.u[0] = sx; m.u[1] = cx; m.u[2] = sy; m.u[3] = cy; m.u[4] = st; m.u[5] = ct;
  return m;
}

// RFF argument a = Omega_f . u of the mapped point and its x, y, t derivatives (om: Omega,
// [F][3] or [F][6], in global or shared memory).
__device__ __forceinline__ float4 rff_arg(const MlpArgs& a, const float* om, const RffMap& m, int f) {
  if (!a.period) {
    const float ox = om[3 * f], oy = om[3 * f + 1], ot = om[3 * f + 2];
    return make_float4(ox * m.u[0] + oy * m.u[1] + ot * m.u[2], ox, oy, ot);
  }
  const float* o = om + 6 * f;
  const float pi = 3.14159265358979f;
  const float o0 = o[0], o1 = o[1], o2 = o[2], o3 = o[3], o4 = o[4], o5 = o[5];
  const float sx = m.u[0], cx = m.u[1], sy = m.u[2], cy = m.u[3], st = m.u[4], ct = m.u[5];
  return make_float4(o0 * sx + o1 * cx + o2 * sy + o3 * cy + o4 * st + o5 * ct, pi * (o0 * cx - o1 * sx),
                     pi * (o2 * cy - o3 * sy), m.w * (o4 * ct - o5 * st));
}

// d/dT of the four rows of both RFF features of frequency f of a mapped point (periodic map):
// T enters through phi = 2 pi t / T in u4 = sin phi, u5 = cos phi and in their t-derivatives.
// dc: the cosine feature's rows (cos a, -sin a da_d), ds: the sine feature's (sin a, cos a da_d).
__device__ __forceinline__ void rff_dfeatures_dT(const MlpArgs& a, const float* om, const RffMap& m, int f,
                                                 float4& dc, float4& ds) {
  const float4 g = rff_arg(a, om, m, f);
  const float w = m.w, st = m.u[4], ct = m.u[5], dphi = m.dphi;   // dphi = d phi / dT
  const float o4 = om[6 * f + 4], o5 = om[6 * f + 5];
  const float daT = o4 * ct * dphi - o5 * st * dphi;           // d a / dT
  const float ddtT = -m.wT * (o4 * ct - o5 * st) + w * (-o4 * st - o5 * ct) * dphi;   // d (da/dt) / dT
  float sn, cs;
  sincosf(g.x, &sn, &cs);
  dc = make_float4(-sn * daT, -cs * daT * g.y, -cs * daT * g.z, -cs * daT * g.w - sn * ddtT);
  ds = make_float4(cs * daT, -sn * daT * g.y, -sn * daT * g.z, -sn * daT * g.w + cs * ddtT);
}

// Warps of the grid walking points: warp index and count.
__device__ __forceinline__ int64_t warp_id_global() { return (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t warp_count_global() { return (gridDim.x * (int64_t)blockDim.x) >> 5; }

// Row buffers are walked as (point, group of four columns): e -> (p, q), the group's columns
// 4q .. 4q + 3 of all four rows of point p.
__device__ __forceinline__ void split_pq(int64_t e, int ng, int64_t& p, int& q) {
  p = e / ng;
  q = (int)(e - p * ng);
}

// The layers' weight matrices copied for the library GEMMs as [outp][ld] (out and in rounded
// up to four, pads zero) at 256-byte aligned offsets; a non-finite weight sets the call's status
// (the GEMMs are FP32 emulated on the tensor cores without special-value handling, so a NaN
// or infinity would not reach the loss by itself).
constexpr int MLP_MAX_LAYERS = 9;
struct MlpCopyArgs {
  const float* src;                  // the premap's trainable parameters
  float* dst;
  int64_t src_off[MLP_MAX_LAYERS], dst_off[MLP_MAX_LAYERS];
  int32_t in[MLP_MAX_LAYERS], ld[MLP_MAX_LAYERS], out[MLP_MAX_LAYERS], outp[MLP_MAX_LAYERS];
  int32_t nl;
  int32_t* status;
};
__global__ void mlp_wcopy_kernel(MlpCopyArgs a) {
  bool bad = false;
  for (int l = 0; l < a.nl; ++l) {
    const int in = a.in[l], ld = a.ld[l];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)a.outp[l] * ld;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t o = e / ld;
      const int i = (int)(e - o * ld);
      float v = 0.f;
      if (i < in && o < a.out[l]) {
        v = a.src[a.src_off[l] + o * in + i];
        bad |= !isfinite(v);
      }
      a.dst[a.dst_off[l] + e] = v;
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(a.status, 0, 5);   // QP_ERR_NONFINITE
}

// RFF features of every point into X (rows by mlp_row): row s = 0 the features (cos of the
// first F columns, sin of the next F), s = 1..3 their tangents (four-row points); pads zeroed.
// One warp per point (the input map once per lane), lanes over the frequencies; Omega in
// shared memory ([F][3] or [F][6] floats).
__global__ void mlp_features_kernel(MlpArgs a, float* X, int ld) {
  extern __shared__ float om[];
  const int F = a.F, lane = threadIdx.x & 31, no = F * (a.period ? 6 : 3);
  for (int e = threadIdx.x; e < no; e += blockDim.x) om[e] = __ldg(&a.omega[e]);
  __syncthreads();
  for (int64_t gp = warp_id_global(); gp < a.ptot; gp += warp_count_global()) {
    int set;
    const RffMap m = rff_map(a, mlp_point(a, gp, set));
    float* r = X + mlp_row(gp, a.n4) * (int64_t)ld;
    const int nr = gp < a.n4 ? 4 : 1;
    for (int f = lane; f < F; f += 32) {
      const float4 g = rff_arg(a, om, m, f);
      float sn, cs;
      sincosf(g.x, &sn, &cs);
      r[f] = cs; r[F + f] = sn;
      if (nr == 4) {
        r[ld + f] = -sn * g.y; r[ld + F + f] = cs * g.y;
        r[2 * ld + f] = -sn * g.z; r[2 * ld + F + f] = cs * g.z;
        r[3 * ld + f] = -sn * g.w; r[3 * ld + F + f] = cs * g.w;
      }
    }
    for (int k = 2 * F + lane; k < ld; k += 32)
      for (int d = 0; d < nr; ++d) r[d * ld + k] = 0.f;
  }
}

// Hidden layer after its contraction, in place on H (rows by mlp_row; pre-activations h0 - b
// and pre-tangents z_d): y0 = tanh(h0), y_d = (1 - y0^2) z_d, four columns per thread.
__global__ void mlp_act_kernel(float* H, const float* b, int64_t P, int out, int ld, int64_t n4) {
  const int ng = ld >> 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P * ng; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p;
    int q;
    split_pq(e, ng, p, q);
    float4* r = reinterpret_cast<float4*>(H + mlp_row(p, n4) * (int64_t)ld) + q;
    const int o = 4 * q;
    const float4 bb = make_float4(o < out ? __ldg(&b[o]) : 0.f, o + 1 < out ? __ldg(&b[o + 1]) : 0.f,
                                  o + 2 < out ? __ldg(&b[o + 2]) : 0.f, o + 3 < out ? __ldg(&b[o + 3]) : 0.f);
    float4 h = r[0];
    h.x = tanhf(h.x + bb.x); h.y = tanhf(h.y + bb.y); h.z = tanhf(h.z + bb.z); h.w = tanhf(h.w + bb.w);
    const float4 sd = make_float4(1.f - h.x * h.x, 1.f - h.y * h.y, 1.f - h.z * h.z, 1.f - h.w * h.w);
    r[0] = h;
#pragma unroll
    for (int d = 1; d < 4; ++d) {
      if (p >= n4) break;
      float4 z = r[d * ng];
      z.x *= sd.x; z.y *= sd.y; z.z *= sd.z; z.w *= sd.w;
      r[d * ng] = z;
    }
  }
}

// Output layer after its contraction (H = [P][4][a.ldo]): theta = g(h), J_d = g'(h) h_d
// (Eq. 27), the rows (h, h_d) kept for the backward, and the dielectric-set count of the loss.
__global__ void mlp_out_kernel(const float* H, MlpArgs a) {
  const int n = a.out, ld = a.ldo;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.ptot * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gp = e / n;
    const int o = (int)(e - gp * n);
    const float* r = H + mlp_row(gp, a.n4) * (int64_t)ld + o;
    const float h = r[0] + __ldg(&a.b[o]);
    const bool tg = gp < a.n4;
    const float hx = tg ? r[ld] : 0.f, hy = tg ? r[2 * ld] : 0.f, ht = tg ? r[3 * ld] : 0.f;
    float g0, g1, g2;
    qpk::scale_tanh(a.scale, h, g0, g1, g2);
    reinterpret_cast<float4*>(a.thetaJ)[e] = make_float4(g0, g1 * hx, g1 * hy, g1 * ht);
    reinterpret_cast<float4*>(a.hout)[e] = make_float4(h, hx, hy, ht);
    if (o == 0 && a.medium == 1) {
      int set;
      const float* v = mlp_point(a, gp, set);
      if (set == 0) {
        const float dx = v[0] - a.disk_x0, dy = v[1] - a.disk_y0;
        if (__fmaf_rn(dx, dx, dy * dy) < a.disk_r * a.disk_r) atomicAdd(&a.counts[0], 1);
      }
    }
  }
}

// Output layer backward, per (point, qubit): cotangents of (h, h_x, h_y, h_t) from dL/dtheta,
// dL/dJ_d, into cot = [P][4][ld] (pad columns zero).
__global__ void mlp_bwd_out_kernel(const float* hout, const float* dthetaJ, int64_t ptot, int n, int ld, int scale,
                                   float* cot, int64_t n4) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ptot * ld; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / ld;
    const int j = (int)(e - p * ld);
    float* c = cot + mlp_row(p, n4) * (int64_t)ld + j;
    const bool tg = p < n4;
    if (j >= n) {
      c[0] = 0.f;
      if (tg) c[ld] = c[2 * ld] = c[3 * ld] = 0.f;
      continue;
    }
    const int64_t en = p * n + j;
    const float4 h = reinterpret_cast<const float4*>(hout)[en];
    const float4 d = reinterpret_cast<const float4*>(dthetaJ)[en];
    float g0, g1, g2;
    qpk::scale_tanh(scale, h.x, g0, g1, g2);
    c[0] = g1 * d.x + g2 * (h.y * d.y + h.z * d.z + h.w * d.w);
    if (tg) {
      c[ld] = g1 * d.y;
      c[2 * ld] = g1 * d.z;
      c[3 * ld] = g1 * d.w;
    }
  }
}

// Through a hidden layer's tanh, in place on dU = [P][4][ld] (cotangents of its outputs y0,
// y_d) with its stored outputs act = [P][4][ld]: dH0 = s dU0 - 2 y0 sum_d y_d dU_d,
// dZ_d = s dU_d, four columns per thread.
__global__ void mlp_dact_kernel(float* dU, const float* act, int64_t P, int ld, int64_t n4) {
  const int ng = ld >> 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P * ng; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p;
    int q;
    split_pq(e, ng, p, q);
    float4* u = reinterpret_cast<float4*>(dU + mlp_row(p, n4) * (int64_t)ld) + q;
    const float4* y = reinterpret_cast<const float4*>(act + mlp_row(p, n4) * (int64_t)ld) + q;
    if (p >= n4) {
      // one-row point: dH0 = s dU0
      const float4 y0 = y[0], u0 = u[0];
      u[0] = make_float4((1.f - y0.x * y0.x) * u0.x, (1.f - y0.y * y0.y) * u0.y, (1.f - y0.z * y0.z) * u0.z,
                         (1.f - y0.w * y0.w) * u0.w);
      continue;
    }
    const float4 y0 = y[0], y1 = y[ng], y2 = y[2 * ng], y3 = y[3 * ng];
    const float4 u0 = u[0];
    float4 u1 = u[ng], u2 = u[2 * ng], u3 = u[3 * ng];
    float4 h;
    h.x = (1.f - y0.x * y0.x) * u0.x - 2.f * y0.x * (y1.x * u1.x + y2.x * u2.x + y3.x * u3.x);
    h.y = (1.f - y0.y * y0.y) * u0.y - 2.f * y0.y * (y1.y * u1.y + y2.y * u2.y + y3.y * u3.y);
    h.z = (1.f - y0.z * y0.z) * u0.z - 2.f * y0.z * (y1.z * u1.z + y2.z * u2.z + y3.z * u3.z);
    h.w = (1.f - y0.w * y0.w) * u0.w - 2.f * y0.w * (y1.w * u1.w + y2.w * u2.w + y3.w * u3.w);
    const float4 sd = make_float4(1.f - y0.x * y0.x, 1.f - y0.y * y0.y, 1.f - y0.z * y0.z, 1.f - y0.w * y0.w);
    u1.x *= sd.x; u1.y *= sd.y; u1.z *= sd.z; u1.w *= sd.w;
    u2.x *= sd.x; u2.y *= sd.y; u2.z *= sd.z; u2.w *= sd.w;
    u3.x *= sd.x; u3.y *= sd.y; u3.z *= sd.z; u3.w *= sd.w;
    u[0] = h;
    u[ng] = u1;
    u[2 * ng] = u2;
    u[3 * ng] = u3;
  }
}

// Bias gradient of one layer per point chunk: slot c gets the sum over the chunk's points of
// the value-row cotangents cot[p][0][o] (0 for chunks past the points). 512 threads: 64
// columns x 8 point lanes, summed in shared memory.
constexpr int DB_THREADS = 512;
__global__ void __launch_bounds__(DB_THREADS) mlp_db_kernel(const float* cot, int64_t P, int out, int ld,
                                                           int64_t chunk, float* part, int64_t nW, int64_t b_off,
                                                           int64_t n4) {
  __shared__ float red[8][64];
  const int c = blockIdx.x, ol = threadIdx.x & 63, j = threadIdx.x >> 6;
  const int64_t p0 = (int64_t)c * chunk, p1 = p0 + chunk < P ? p0 + chunk : P;
  for (int o0 = 0; o0 < out; o0 += 64) {
    const int o = o0 + ol;
    float acc = 0.f;
    if (o < out)
      for (int64_t p = p0 + j; p < p1; p += 8) acc += cot[mlp_row(p, n4) * (int64_t)ld + o];
    red[j][ol] = acc;
    __syncthreads();
    if (j == 0 && o < out) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) t += red[k][ol];
      part[(int64_t)c * nW + b_off + o] = t;
    }
    __syncthreads();
  }
}

// One layer's per-chunk dW (column-major in x out with leading dimension ldw, one scratch row
// of stride dws per chunk) into the parameter segment [off, off + out * in) of every partial
// slot as row-major [out][in]: slots c < used take their chunk's dW, the others 0.
__global__ void mlp_dw_slots_kernel(const float* dw, int64_t dws, int ldw, float* part, int64_t nW, int64_t off,
                                    int in, int out, int used, int nchunks) {
  const int64_t len = (int64_t)out * in, tot = (int64_t)nchunks * len;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / len, k = e - c * len;
    const int64_t o = k / in, i = k - o * in;
    part[c * nW + off + k] = c < used ? dw[c * dws + o * ldw + i] : 0.f;
  }
}

// Learned period's gradient from the first layer's input cotangents dX = [P][4][ld]: the sum
// over points and features of dX . d(features)/dT, one warp per point (the input map once per
// lane), lanes over the frequencies (both features of one), added in FP64. The cotangents of
// four frequencies per lane are loaded before any is used; Omega ([F][6]) in shared memory.
__global__ void mlp_period_kernel(const float* dX, MlpArgs a, int ld, double* tgrad) {
  extern __shared__ float om[];
  const int F = a.F, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < 6 * F; e += blockDim.x) om[e] = __ldg(&a.omega[e]);
  __syncthreads();
  float tg = 0.f;
  for (int64_t gp = warp_id_global(); gp < a.ptot; gp += warp_count_global()) {
    int set;
    const RffMap m = rff_map(a, mlp_point(a, gp, set));
    const float* r = dX + mlp_row(gp, a.n4) * (int64_t)ld;
    const int nr = gp < a.n4 ? 4 : 1;
    for (int f0 = 0; f0 < F; f0 += 128) {
      float x[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int f = f0 + lane + 32 * i;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          x[i][d] = f < F && d < nr ? r[d * ld + f] : 0.f;
          x[i][4 + d] = f < F && d < nr ? r[d * ld + F + f] : 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int f = f0 + lane + 32 * i;
        if (f >= F) continue;
        float4 dc, ds;
        rff_dfeatures_dT(a, om, m, f, dc, ds);
        tg += x[i][0] * dc.x + x[i][1] * dc.y + x[i][2] * dc.z + x[i][3] * dc.w;
        tg += x[i][4] * ds.x + x[i][5] * ds.y + x[i][6] * ds.z + x[i][7] * ds.w;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tg += __shfl_xor_sync(0xffffffffu, tg, o);
  if (lane == 0) atomicAdd(tgrad, (double)tg);
}

// The learned period's gradient into the weight-gradient partial slots: chunk 0 takes the sum,
// the others 0 (the reduction adds all chunks).
__global__ void mlp_period_fin_kernel(const double* tgrad, float* part, int64_t nW, int64_t t_off, int nchunks) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nchunks; b += gridDim.x * blockDim.x)
    part[(int64_t)b * nW + t_off] = b == 0 ? (float)*tgrad : 0.f;
}

// ------------------------------------------------------------------- fused output layer
// Warp reduce-scatter of 32 values per lane: afterwards v[0] of lane L is the warp's sum of
// value L (each halving step keeps the half of the values that the lane's bit selects).
__device__ __forceinline__ void warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float keep = up ? v[i + h] : v[i], send = up ? v[i] : v[i + h];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
}

// The output layer has only n (<= 16) units, too narrow for a GEMM to pay: its contraction is
// done per point inside the kernels that already pass over the last hidden layer's rows.
// Forward: the last hidden layer's activation (in place on its pre-activation rows) and the
// output layer (h_j,s = sum_k W_jk y_s,k) with the scaling, one warp per point, lane q on
// hidden units 4q .. 4q + 3 (at most 128 units); W in shared memory as [n][ld]. The next
// point's rows are loaded while the current one is worked on.
// a: the output layer (W, b, in = H, out = n, ldi = row stride of the hidden rows).
template <int NMAX>
__global__ void __launch_bounds__(256) mlp_act_out_kernel(MlpArgs a, float* Hh, const float* bh) {
  extern __shared__ float4 wsm4[];
  float* wsm = reinterpret_cast<float*>(wsm4);
  const int n = a.out, H = a.in, ld = a.ldi, ng = ld >> 2, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < n * ld; e += blockDim.x) {
    const int j = e / ld, k = e - j * ld;
    wsm[e] = k < H ? __ldg(&a.W[j * H + k]) : 0.f;
  }
  __syncthreads();
  const bool active = lane < ng;
  const int q = lane, o = 4 * q;
  const float4 bb = make_float4(o < H ? __ldg(&bh[o]) : 0.f, o + 1 < H ? __ldg(&bh[o + 1]) : 0.f,
                                o + 2 < H ? __ldg(&bh[o + 2]) : 0.f, o + 3 < H ? __ldg(&bh[o + 3]) : 0.f);
  const int64_t nw = warp_count_global();
  float4 yn[4];
  int64_t gp = warp_id_global();
  {
    const int nr = gp < a.n4 ? 4 : 1;
#pragma unroll
    for (int d = 0; d < 4; ++d)
      yn[d] = active && d < nr && gp < a.ptot
                  ? reinterpret_cast<const float4*>(Hh + mlp_row(gp, a.n4) * (int64_t)ld)[d * ng + q]
                  : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (; gp < a.ptot; gp += nw) {
    float acc[NMAX][4];
#pragma unroll
    for (int j = 0; j < NMAX; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    float4* r = reinterpret_cast<float4*>(Hh + mlp_row(gp, a.n4) * (int64_t)ld);
    const int rpp = gp < a.n4 ? 4 : 1;
    float4 y[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) y[d] = yn[d];
    if (active && gp + nw < a.ptot) {
      const float4* rn = reinterpret_cast<const float4*>(Hh + mlp_row(gp + nw, a.n4) * (int64_t)ld);
      const int nrn = gp + nw < a.n4 ? 4 : 1;
#pragma unroll
      for (int d = 0; d < 4; ++d) yn[d] = d < nrn ? rn[d * ng + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (active) {
      y[0].x = tanhf(y[0].x + bb.x); y[0].y = tanhf(y[0].y + bb.y);
      y[0].z = tanhf(y[0].z + bb.z); y[0].w = tanhf(y[0].w + bb.w);
      const float4 sd = make_float4(1.f - y[0].x * y[0].x, 1.f - y[0].y * y[0].y, 1.f - y[0].z * y[0].z,
                                    1.f - y[0].w * y[0].w);
#pragma unroll
      for (int d = 1; d < 4; ++d) { y[d].x *= sd.x; y[d].y *= sd.y; y[d].z *= sd.z; y[d].w *= sd.w; }
#pragma unroll
      for (int d = 0; d < 4; ++d)
        if (d < rpp) r[d * ng + q] = y[d];
#pragma unroll
      for (int j = 0; j < NMAX; ++j) {
        if (j >= n) break;
        const float4 w = wsm4[j * ng + q];
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[j][d] = w.x * y[d].x + w.y * y[d].y + w.z * y[d].z + w.w * y[d].w;
      }
    }
    // warp sums by reduce-scatter over groups of eight units: afterwards lane 4j' + d holds
    // row d of unit 8g + j' of group g
#pragma unroll
    for (int g = 0; g < NMAX / 8; ++g) {
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = acc[8 * g + (i >> 2)][i & 3];
      warp_reduce_scatter32(v, lane);
      const float h1 = __shfl_down_sync(0xffffffffu, v[0], 1), h2 = __shfl_down_sync(0xffffffffu, v[0], 2),
                  h3 = __shfl_down_sync(0xffffffffu, v[0], 3);
      const int j = 8 * g + (lane >> 2);
      if ((lane & 3) == 0 && j < n) {
        const int64_t e = gp * n + j;
        const float h0 = v[0] + __ldg(&a.b[j]);
        float g0, g1, g2;
        qpk::scale_tanh(a.scale, h0, g0, g1, g2);
        reinterpret_cast<float4*>(a.thetaJ)[e] = make_float4(g0, g1 * h1, g1 * h2, g1 * h3);
        reinterpret_cast<float4*>(a.hout)[e] = make_float4(h0, h1, h2, h3);
      }
    }
    if (lane == 0 && a.medium == 1) {
      int set;
      const float* v = mlp_point(a, gp, set);
      if (set == 0) {
        const float dx = v[0] - a.disk_x0, dy = v[1] - a.disk_y0;
        if (__fmaf_rn(dx, dx, dy * dy) < a.disk_r * a.disk_r) atomicAdd(&a.counts[0], 1);
      }
    }
  }
}

// Backward through the output layer and the last hidden layer's tanh, per point chunk (block
// c = weight-gradient slot c): the output cotangents c_j,s from dL/dtheta, dL/dJ (Eq. 27
// chain rule), dU_s = sum_j c_j,s W_j (the hidden outputs' cotangents), then the tanh backward
// into cot = [P][4][ld] (pad columns zero); the output layer's dW_jk = sum_p,s c_j,s y_s,k and
// db_j = sum_p c_j,0 accumulated per lane, summed over the block in shared memory and written
// to slot c. One warp per point, lanes over groups of four hidden units (ld <= 128).
template <int NMAX>
__global__ void __launch_bounds__(256, 2) mlp_out_bwd_kernel(MlpArgs a, const float* hout, const float* dthetaJ,
                                                          const float* act, float* cot, int64_t chunk, float* part,
                                                          int64_t nW, int64_t w_off, int64_t b_off) {
  extern __shared__ float4 osm4[];
  const int n = a.out, H = a.in, ld = a.ldi, ng = ld >> 2, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  float* wsm = reinterpret_cast<float*>(osm4);   // [n][ld] weights
  float* dws = wsm + n * ld;                     // [n][ld] block's dW
  float* dbs = dws + n * ld;                     // [n] block's db
  for (int e = threadIdx.x; e < n * ld; e += blockDim.x) {
    const int j = e / ld, k = e - j * ld;
    wsm[e] = k < H ? __ldg(&a.W[j * H + k]) : 0.f;
    dws[e] = 0.f;
  }
  if (threadIdx.x < n) dbs[threadIdx.x] = 0.f;
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * chunk;
  const int64_t p1 = p0 + chunk < a.ptot ? p0 + chunk : a.ptot;
  float4 dwacc[NMAX];
#pragma unroll
  for (int j = 0; j < NMAX; ++j) dwacc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  float dbacc = 0.f;
  const bool active = lane < ng;
  // the next point's rows are loaded while the current one is worked on
  float4 yn[4], hn = make_float4(0.f, 0.f, 0.f, 0.f), dn = hn;
  {
    const int64_t gp = p0 + warp;
    const float4* y4 = reinterpret_cast<const float4*>(act + mlp_row(gp, a.n4) * (int64_t)ld);
    const int nr = gp < a.n4 ? 4 : 1;
#pragma unroll
    for (int d = 0; d < 4; ++d)
      yn[d] = active && gp < p1 && d < nr ? y4[d * ng + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < n && gp < p1) {
      hn = reinterpret_cast<const float4*>(hout)[gp * n + lane];
      dn = reinterpret_cast<const float4*>(dthetaJ)[gp * n + lane];
    }
  }
  for (int64_t gp = p0 + warp; gp < p1; gp += nwarp) {
    float4 y[4], u[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      y[d] = yn[d];
      u[d] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float4 h = hn, d = dn;
    if (gp + nwarp < p1) {
      const int64_t g2 = gp + nwarp;
      const float4* y4 = reinterpret_cast<const float4*>(act + mlp_row(g2, a.n4) * (int64_t)ld);
      const int nr2 = g2 < a.n4 ? 4 : 1;
      if (active) {
#pragma unroll
        for (int k = 0; k < 4; ++k) yn[k] = k < nr2 ? y4[k * ng + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (lane < n) {
        hn = reinterpret_cast<const float4*>(hout)[g2 * n + lane];
        dn = reinterpret_cast<const float4*>(dthetaJ)[g2 * n + lane];
      }
    }
    // output cotangents: lane j < n holds unit j's four rows
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    if (lane < n) {
      float g0, g1, g2;
      qpk::scale_tanh(a.scale, h.x, g0, g1, g2);
      c[0] = g1 * d.x + g2 * (h.y * d.y + h.z * d.z + h.w * d.w);
      c[1] = g1 * d.y;
      c[2] = g1 * d.z;
      c[3] = g1 * d.w;
      dbacc += c[0];
    }
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      if (j >= n) break;
      float cj[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) cj[d] = __shfl_sync(0xffffffffu, c[d], j);
      const float4 w = active ? osm4[j * ng + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        u[d].x += cj[d] * w.x; u[d].y += cj[d] * w.y; u[d].z += cj[d] * w.z; u[d].w += cj[d] * w.w;
        dwacc[j].x += cj[d] * y[d].x; dwacc[j].y += cj[d] * y[d].y;
        dwacc[j].z += cj[d] * y[d].z; dwacc[j].w += cj[d] * y[d].w;
      }
    }
    if (active) {
      // tanh backward: dH0 = s dU0 - 2 y0 sum_d y_d dU_d, dZ_d = s dU_d
      float4* c4 = reinterpret_cast<float4*>(cot + mlp_row(gp, a.n4) * (int64_t)ld);
      const float4 sd = make_float4(1.f - y[0].x * y[0].x, 1.f - y[0].y * y[0].y, 1.f - y[0].z * y[0].z,
                                    1.f - y[0].w * y[0].w);
      float4 h0;
      h0.x = sd.x * u[0].x - 2.f * y[0].x * (y[1].x * u[1].x + y[2].x * u[2].x + y[3].x * u[3].x);
      h0.y = sd.y * u[0].y - 2.f * y[0].y * (y[1].y * u[1].y + y[2].y * u[2].y + y[3].y * u[3].y);
      h0.z = sd.z * u[0].z - 2.f * y[0].z * (y[1].z * u[1].z + y[2].z * u[2].z + y[3].z * u[3].z);
      h0.w = sd.w * u[0].w - 2.f * y[0].w * (y[1].w * u[1].w + y[2].w * u[2].w + y[3].w * u[3].w);
      c4[lane] = h0;
      if (gp < a.n4) {
#pragma unroll
        for (int d = 1; d < 4; ++d)
          c4[d * ng + lane] = make_float4(sd.x * u[d].x, sd.y * u[d].y, sd.z * u[d].z, sd.w * u[d].w);
      }
    }
  }
  // block sums of dW and db, then the slot
  if (active) {
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      if (j >= n) break;
      float* d = dws + j * ld + 4 * lane;
      atomicAdd(d, dwacc[j].x); atomicAdd(d + 1, dwacc[j].y); atomicAdd(d + 2, dwacc[j].z); atomicAdd(d + 3, dwacc[j].w);
    }
  }
  if (lane < n) atomicAdd(&dbs[lane], dbacc);
  __syncthreads();
  float* slot = part + (int64_t)blockIdx.x * nW;
  for (int e = threadIdx.x; e < n * H; e += blockDim.x) {
    const int j = e / H, k = e - j * H;
    slot[w_off + e] = dws[j * ld + k];
  }
  if (threadIdx.x < n) slot[b_off + threadIdx.x] = dbs[threadIdx.x];
}

}  // namespace qpm
