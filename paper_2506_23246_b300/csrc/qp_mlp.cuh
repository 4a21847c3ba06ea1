// qp_mlp.cuh -- the RFF + tanh MLP premap of any depth and width (Sec. 2.2 architecture: RFF
// features, fully connected tanh layers, a linear layer to one angle per qubit, Eq. 27
// scaling), forward with its input tangents and backward with the weight gradients.
//
// Every point carries four rows through the network: the value and its derivatives along x, y
// and t (forward-mode tangents). For a tanh layer with pre-activation h = W u + b the rows are
//   y0 = tanh(h0),  y_d = s z_d  with  s = 1 - y0^2,  z_d = W u_d  (the pre-tangents),
// and the layer stores (y0, z_x, z_y, z_t) per unit. Its backward, from the cotangents dU of
// (y0, y_d), is
//   dH0 = s dU0 - 2 y0 s sum_d z_d dU_d,   dZ_d = s dU_d,
//   dW += dH0 u0^T + sum_d dZ_d u_d^T,  db += dH0,   dU_prev = W^T (dH0 | dZ_d).
// The first layer's input is r = [cos(Omega v), sin(Omega v)] with tangents
// [-sin(Omega v) Omega_d, cos(Omega v) Omega_d], computed where it is loaded. The output layer
// gives theta = g(h), J_d = g'(h) h_d (Eq. 27 on a = tanh(h)); its backward is
//   dH = g'(h) dtheta + g''(h) sum_d h_d dJ_d,   dH_d = g'(h) dJ_d.
//
// The contractions are tiled FP32 SIMT GEMMs: a tile of 32 points (128 rows, the four rows of
// a point in one thread) x 64 outputs, K in slices of 32 through shared memory; the epilogues
// couple a point's four rows (tanh and its derivative). The weight gradients reduce over rows
// in row chunks, one partial per chunk summed later in FP64.
#pragma once
#include <cuda_runtime.h>

#include "qp_common.h"
#include "qp_aux.cuh"

namespace qpm {

constexpr int MT_P = 32;        // points per tile (128 rows)
constexpr int MT_N = 64;        // outputs per tile
constexpr int MT_K = 32;        // K slice
constexpr int MT_THREADS = 256;

struct MlpArgs {
  // points of the call (three sets in order), global point index gp = set base + local index
  const float* pts[3];
  int64_t npts[3];
  int64_t ptot;
  const float* omega;       // [F][3], or [F][6] with the periodic map (fixed RFF frequencies)
  int32_t F;
  const float* period;      // periodic input map (Eqs. 25-26): the learned time period T, or null
  // the layer: out x in weights (row-major [out][in]) and bias
  const float* W;
  const float* b;
  int32_t in, out;
  int32_t in_rff;           // 1: the input is the RFF features (in = 2F), 0: the previous layer
  const float* act_in;      // previous layer's (y0, z_x, z_y, z_t) [P][4][in] (in_rff = 0)
  // forward outputs
  float* act_out;           // hidden layer: [P][4][out]
  int32_t final_layer;      // 1: output layer -> theta, J (thetaJ) and h (hout)
  int32_t scale;            // Eq. 27 scaling of the output layer
  float* thetaJ;            // [P][out] float4
  float* hout;              // [P][out] float4 (h, h_x, h_y, h_t)
  // dielectric-set count of the loss (output layer of the forward)
  int32_t* counts;
  int32_t medium;
  float disk_r, disk_x0, disk_y0;
};

__device__ __forceinline__ const float* mlp_point(const MlpArgs& a, int64_t gp, int& set) {
  set = 0;
  int64_t li = gp;
  if (li >= a.npts[0]) { li -= a.npts[0]; set = 1; if (li >= a.npts[1]) { li -= a.npts[1]; set = 2; } }
  return a.pts[set] + li * 3;
}

// RFF argument a = Omega_f . u(v) of point v and its x, y, t derivatives: u = v, or with the
// periodic map (Eqs. 25-26) u = (sin pi x, cos pi x, sin pi y, cos pi y, sin(2 pi t/T),
// cos(2 pi t/T)).
__device__ __forceinline__ float4 rff_arg(const MlpArgs& a, const float* v, int f) {
  if (!a.period) {
    const float ox = __ldg(&a.omega[3 * f]), oy = __ldg(&a.omega[3 * f + 1]), ot = __ldg(&a.omega[3 * f + 2]);
    return make_float4(ox * v[0] + oy * v[1] + ot * v[2], ox, oy, ot);
  }
  const float* o = a.omega + 6 * f;
  const float T = __ldg(a.period), w = 6.28318530717959f / T;
  float sx, cx, sy, cy, st, ct;
  sincospif(v[0], &sx, &cx);
  sincospif(v[1], &sy, &cy);
  sincosf(w * v[2], &st, &ct);
  const float pi = 3.14159265358979f;
  const float o0 = __ldg(o), o1 = __ldg(o + 1), o2 = __ldg(o + 2), o3 = __ldg(o + 3), o4 = __ldg(o + 4), o5 = __ldg(o + 5);
  return make_float4(o0 * sx + o1 * cx + o2 * sy + o3 * cy + o4 * st + o5 * ct, pi * (o0 * cx - o1 * sx),
                     pi * (o2 * cy - o3 * sy), w * (o4 * ct - o5 * st));
}

// Input rows of point gp at input index k (< in), all four: RFF features and their tangents,
// or the previous layer's (y0, s z_d).
__device__ __forceinline__ float4 mlp_input(const MlpArgs& a, int64_t gp, int k) {
  if (gp >= a.ptot) return make_float4(0.f, 0.f, 0.f, 0.f);
  if (a.in_rff) {
    int set;
    const float* v = mlp_point(a, gp, set);
    const int f = k < a.F ? k : k - a.F;
    const float4 g = rff_arg(a, v, f);
    float sn, cs;
    sincosf(g.x, &sn, &cs);
    const float val = k < a.F ? cs : sn, d = k < a.F ? -sn : cs;
    return make_float4(val, d * g.y, d * g.z, d * g.w);
  }
  const float* r = a.act_in + gp * 4 * (int64_t)a.in + k;
  const float y0 = r[0], sd = 1.f - y0 * y0;
  return make_float4(y0, sd * r[a.in], sd * r[2 * a.in], sd * r[3 * a.in]);
}

// Forward of one layer: C = X W^T (+ b on the value row), then tanh (hidden) or the scaling
// (output layer).
__global__ void __launch_bounds__(MT_THREADS) mlp_fwd_kernel(MlpArgs a) {
  __shared__ float xs[MT_K][MT_P * 4 + 4];   // [k][point * 4 + row]
  __shared__ float ws[MT_K][MT_N + 4];       // [k][output]
  const int tid = threadIdx.x, tp = tid >> 4, to = tid & 15;
  const int64_t ntile_p = (a.ptot + MT_P - 1) / MT_P;
  const int ntile_n = (a.out + MT_N - 1) / MT_N;
  for (int64_t t = blockIdx.x; t < ntile_p * ntile_n; t += gridDim.x) {
    const int64_t p0 = (t / ntile_n) * MT_P;
    const int n0 = (int)(t % ntile_n) * MT_N;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][s][j] = 0.f;
    for (int k0 = 0; k0 < a.in; k0 += MT_K) {
      __syncthreads();
      for (int e = tid; e < MT_P * MT_K; e += MT_THREADS) {
        const int pl = e / MT_K, kk = e % MT_K;
        const float4 x = (k0 + kk < a.in) ? mlp_input(a, p0 + pl, k0 + kk) : make_float4(0.f, 0.f, 0.f, 0.f);
        xs[kk][pl * 4 + 0] = x.x; xs[kk][pl * 4 + 1] = x.y; xs[kk][pl * 4 + 2] = x.z; xs[kk][pl * 4 + 3] = x.w;
      }
      for (int e = tid; e < MT_N * MT_K; e += MT_THREADS) {
        const int o = e / MT_K, kk = e % MT_K;
        ws[kk][o] = (n0 + o < a.out && k0 + kk < a.in) ? __ldg(&a.W[(int64_t)(n0 + o) * a.in + k0 + kk]) : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < MT_K; ++kk) {
        const float4 x0 = *reinterpret_cast<const float4*>(&xs[kk][(tp * 2) * 4]);
        const float4 x1 = *reinterpret_cast<const float4*>(&xs[kk][(tp * 2 + 1) * 4]);
        const float4 w = *reinterpret_cast<const float4*>(&ws[kk][to * 4]);
        const float xv[2][4] = {{x0.x, x0.y, x0.z, x0.w}, {x1.x, x1.y, x1.z, x1.w}};
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][s][j] = fmaf(xv[i][s], wv[j], acc[i][s][j]);
      }
    }
    // epilogue: a point's four rows are this thread's
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int64_t gp = p0 + tp * 2 + i;
      if (gp >= a.ptot) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int o = n0 + to * 4 + j;
        if (o >= a.out) continue;
        const float h = acc[i][0][j] + __ldg(&a.b[o]);
        if (a.final_layer) {
          float g0, g1, g2;
          qpk::scale_tanh(a.scale, h, g0, g1, g2);
          reinterpret_cast<float4*>(a.thetaJ)[gp * a.out + o] =
              make_float4(g0, g1 * acc[i][1][j], g1 * acc[i][2][j], g1 * acc[i][3][j]);
          reinterpret_cast<float4*>(a.hout)[gp * a.out + o] = make_float4(h, acc[i][1][j], acc[i][2][j], acc[i][3][j]);
        } else {
          float* r = a.act_out + gp * 4 * (int64_t)a.out + o;
          r[0] = tanhf(h);
          r[a.out] = acc[i][1][j];
          r[2 * a.out] = acc[i][2][j];
          r[3 * a.out] = acc[i][3][j];
        }
      }
      if (a.final_layer && n0 == 0 && to == 0 && a.medium == 1) {
        int set;
        const float* v = mlp_point(a, gp, set);
        if (set == 0) {
          const float dx = v[0] - a.disk_x0, dy = v[1] - a.disk_y0;
          if (__fmaf_rn(dx, dx, dy * dy) < a.disk_r * a.disk_r) atomicAdd(&a.counts[0], 1);
        }
      }
    }
  }
}

// Output layer backward, elementwise per (point, qubit): cotangents of (h, h_x, h_y, h_t)
// from dL/dtheta, dL/dJ_d, into cot [P][4][n].
__global__ void mlp_bwd_out_kernel(const float* hout, const float* dthetaJ, int64_t ptot, int n, int scale,
                                   float* cot) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ptot * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / n;
    const int j = (int)(e % n);
    const float4 h = reinterpret_cast<const float4*>(hout)[e];
    const float4 d = reinterpret_cast<const float4*>(dthetaJ)[e];
    float g0, g1, g2;
    qpk::scale_tanh(scale, h.x, g0, g1, g2);
    float* c = cot + p * 4 * (int64_t)n + j;
    c[0] = g1 * d.x + g2 * (h.y * d.y + h.z * d.z + h.w * d.w);
    c[n] = g1 * d.y;
    c[2 * n] = g1 * d.z;
    c[3 * n] = g1 * d.w;
  }
}

struct MlpBwdArgs {
  int64_t ptot;
  const float* W;           // [out][in] weights of the layer whose input cotangents are formed
  int32_t in, out;
  const float* cot;         // [P][4][out] cotangents of the layer's pre-activations
  const float* act_prev;    // [P][4][in] (y0, z) of the previous hidden layer
  float* cot_prev;          // [P][4][in] cotangents of the previous layer's pre-activations
  // first layer with the periodic map: the input cotangents are contracted with the features'
  // derivative by the learned period and summed into *tgrad (FP64) instead of being stored
  MlpArgs x;
  double* tgrad;
};

// d/dT of the four rows of RFF feature k of point v (periodic map): T enters through
// phi = 2 pi t / T in u4 = sin phi, u5 = cos phi and in their t-derivatives.
__device__ __forceinline__ float4 rff_dfeature_dT(const MlpArgs& a, const float* v, int k) {
  const int f = k < a.F ? k : k - a.F;
  const float4 g = rff_arg(a, v, f);
  const float T = __ldg(a.period), w = 6.28318530717959f / T, ph = w * v[2];
  float st, ct;
  sincosf(ph, &st, &ct);
  const float o4 = __ldg(&a.omega[6 * f + 4]), o5 = __ldg(&a.omega[6 * f + 5]);
  const float dphi = -ph / T;                                  // d phi / dT
  const float daT = o4 * ct * dphi - o5 * st * dphi;           // d a / dT
  const float ddtT = -w / T * (o4 * ct - o5 * st) + w * (-o4 * st - o5 * ct) * dphi;   // d (da/dt) / dT
  float sn, cs;
  sincosf(g.x, &sn, &cs);
  if (k < a.F)   // rows: cos a, -sin a da_d
    return make_float4(-sn * daT, -cs * daT * g.y, -cs * daT * g.z, -cs * daT * g.w - sn * ddtT);
  return make_float4(cs * daT, -sn * daT * g.y, -sn * daT * g.z, -sn * daT * g.w + cs * ddtT);
}

// dU = cot W (the cotangents of the previous layer's outputs y0, y_d), then through that
// layer's tanh: cot_prev = (s dU0 - 2 y0 s sum_d z_d dU_d, s dU_d).
__global__ void __launch_bounds__(MT_THREADS) mlp_bwd_dx_kernel(MlpBwdArgs a) {
  __shared__ float cs[MT_K][MT_P * 4 + 4];   // [o][point * 4 + row]
  __shared__ float ws[MT_K][MT_N + 4];       // [o][input index]
  const int tid = threadIdx.x, tp = tid >> 4, to = tid & 15;
  const int64_t ntile_p = (a.ptot + MT_P - 1) / MT_P;
  const int ntile_n = (a.in + MT_N - 1) / MT_N;
  for (int64_t t = blockIdx.x; t < ntile_p * ntile_n; t += gridDim.x) {
    const int64_t p0 = (t / ntile_n) * MT_P;
    const int n0 = (int)(t % ntile_n) * MT_N;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][s][j] = 0.f;
    for (int k0 = 0; k0 < a.out; k0 += MT_K) {
      __syncthreads();
      for (int e = tid; e < MT_P * 4 * MT_K; e += MT_THREADS) {
        const int row = e / MT_K, kk = e % MT_K;   // row = point * 4 + s
        const int64_t gp = p0 + row / 4;
        cs[kk][row] = (gp < a.ptot && k0 + kk < a.out) ? a.cot[(gp * 4 + (row & 3)) * (int64_t)a.out + k0 + kk] : 0.f;
      }
      for (int e = tid; e < MT_N * MT_K; e += MT_THREADS) {
        const int kk = e / MT_N, i = e % MT_N;
        ws[kk][i] = (n0 + i < a.in && k0 + kk < a.out) ? __ldg(&a.W[(int64_t)(k0 + kk) * a.in + n0 + i]) : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < MT_K; ++kk) {
        const float4 c0 = *reinterpret_cast<const float4*>(&cs[kk][(tp * 2) * 4]);
        const float4 c1 = *reinterpret_cast<const float4*>(&cs[kk][(tp * 2 + 1) * 4]);
        const float4 w = *reinterpret_cast<const float4*>(&ws[kk][to * 4]);
        const float cv[2][4] = {{c0.x, c0.y, c0.z, c0.w}, {c1.x, c1.y, c1.z, c1.w}};
        const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][s][j] = fmaf(cv[i][s], wv[j], acc[i][s][j]);
      }
    }
    if (a.tgrad) {
      // periodic map: sum over the tile of dL/dr_s[k] dr_s[k]/dT
      float tg = 0.f;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int64_t gp = p0 + tp * 2 + i;
        if (gp >= a.ptot) continue;
        int set;
        const float* v = mlp_point(a.x, gp, set);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = n0 + to * 4 + j;
          if (k >= a.in) continue;
          const float4 d = rff_dfeature_dT(a.x, v, k);
          tg += acc[i][0][j] * d.x + acc[i][1][j] * d.y + acc[i][2][j] * d.z + acc[i][3][j] * d.w;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tg += __shfl_xor_sync(0xffffffffu, tg, o);
      if ((tid & 31) == 0) atomicAdd(a.tgrad, (double)tg);
      continue;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int64_t gp = p0 + tp * 2 + i;
      if (gp >= a.ptot) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = n0 + to * 4 + j;
        if (k >= a.in) continue;
        const float* r = a.act_prev + gp * 4 * (int64_t)a.in + k;
        const float y0 = r[0], sd = 1.f - y0 * y0;
        const float zs = r[a.in] * acc[i][1][j] + r[2 * a.in] * acc[i][2][j] + r[3 * a.in] * acc[i][3][j];
        float* c = a.cot_prev + gp * 4 * (int64_t)a.in + k;
        c[0] = sd * acc[i][0][j] - 2.f * y0 * sd * zs;
        c[a.in] = sd * acc[i][1][j];
        c[2 * a.in] = sd * acc[i][2][j];
        c[3 * a.in] = sd * acc[i][3][j];
      }
    }
  }
}

struct MlpDwArgs {
  MlpArgs x;                // the layer's input (RFF features or previous layer) and sizes
  const float* cot;         // [P][4][out]
  float* part;              // [nchunks][nW] partial slots of all MLP parameters
  int64_t nW, w_off, b_off; // offsets of this layer's W and b in a slot
  int32_t nchunks;
};

// Weight gradient of one layer over the points of chunk blockIdx.y:
// dW[o][i] = sum_p sum_s cot[p][s][o] x[p][s][i], db[o] = sum_p cot[p][0][o] (blocks of the
// first input tile), written to the chunk's partial slot.
__global__ void __launch_bounds__(MT_THREADS) mlp_dw_kernel(MlpDwArgs a) {
  __shared__ float cs[MT_K][MT_N + 4];   // [row][o]
  __shared__ float xs[MT_K][MT_N + 4];   // [row][i]
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int out = a.x.out, in = a.x.in;
  const int nto = (out + MT_N - 1) / MT_N;
  const int o0 = (blockIdx.x % nto) * MT_N, i0 = (blockIdx.x / nto) * MT_N;
  const int64_t P = a.x.ptot;
  const int64_t pb = P * blockIdx.y / a.nchunks, pe = P * (blockIdx.y + 1) / a.nchunks;
  float acc[4][4], db[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    db[u] = 0.f;
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  }
  // rows in slices of MT_K = 8 points x 4 rows
  for (int64_t r0 = pb * 4; r0 < pe * 4; r0 += MT_K) {
    __syncthreads();
    for (int e = tid; e < MT_K * MT_N; e += MT_THREADS) {
      const int rr = e / MT_N, o = e % MT_N;
      const int64_t row = r0 + rr;
      cs[rr][o] = (row < pe * 4 && o0 + o < out) ? a.cot[row * out + o0 + o] : 0.f;
    }
    for (int e = tid; e < (MT_K / 4) * MT_N; e += MT_THREADS) {
      const int pl = e / MT_N, i = e % MT_N;
      const int64_t gp = r0 / 4 + pl;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gp < pe && i0 + i < in) x = mlp_input(a.x, gp, i0 + i);
      xs[pl * 4 + 0][i] = x.x; xs[pl * 4 + 1][i] = x.y; xs[pl * 4 + 2][i] = x.z; xs[pl * 4 + 3][i] = x.w;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < MT_K; ++rr) {
      const float4 c = *reinterpret_cast<const float4*>(&cs[rr][ty * 4]);
      const float4 x = *reinterpret_cast<const float4*>(&xs[rr][tx * 4]);
      const float cv[4] = {c.x, c.y, c.z, c.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(cv[u], xv[v], acc[u][v]);
      if ((rr & 3) == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) db[u] += cv[u];
      }
    }
  }
  float* slot = a.part + (int64_t)blockIdx.y * a.nW;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int o = o0 + ty * 4 + u;
    if (o >= out) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + tx * 4 + v;
      if (i < in) slot[a.w_off + (int64_t)o * in + i] = acc[u][v];
    }
    if (i0 == 0 && tx == 0) slot[a.b_off + o] = db[u];
  }
}

// The learned period's gradient into the weight-gradient partial slots: chunk 0 takes the sum,
// the others 0 (the reduction adds all chunks).
__global__ void mlp_period_fin_kernel(const double* tgrad, float* part, int64_t nW, int64_t t_off, int nchunks) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nchunks; b += gridDim.x * blockDim.x)
    part[(int64_t)b * nW + t_off] = b == 0 ? (float)*tgrad : 0.f;
}

// ------------------------------------------------------------------------- library-GEMM form
// The layers' contractions as plain GEMMs (library calls on the tensor cores, FP32 results),
// with the point-coupled parts as elementwise kernels around them. Rows are (point, s) with
// s = 0 the value and s = 1..3 the x, y, t tangents; a hidden layer's stored rows are its
// outputs (y0, y_d = s z_d), which are the next layer's inputs as they stand.

// RFF features of every point, [P][4][2F]: row s = 0 the features, s = 1..3 their tangents.
__global__ void mlp_features_kernel(MlpArgs a, float* X) {
  const int F = a.F;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.ptot * F;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gp = e / F;
    const int f = (int)(e % F);
    int set;
    const float* v = mlp_point(a, gp, set);
    const float4 g = rff_arg(a, v, f);
    float sn, cs;
    sincosf(g.x, &sn, &cs);
    float* r = X + gp * 4 * (int64_t)(2 * F);
    r[f] = cs; r[F + f] = sn;
    r[2 * F + f] = -sn * g.y; r[2 * F + F + f] = cs * g.y;
    r[4 * F + f] = -sn * g.z; r[4 * F + F + f] = cs * g.z;
    r[6 * F + f] = -sn * g.w; r[6 * F + F + f] = cs * g.w;
  }
}

// Hidden layer after its contraction, in place on H = [P][4][out] (pre-activations h0 - b and
// pre-tangents z_d): y0 = tanh(h0), y_d = (1 - y0^2) z_d.
__global__ void mlp_act_kernel(float* H, const float* b, int64_t P, int out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P * out; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / out;
    const int o = (int)(e % out);
    float* r = H + p * 4 * (int64_t)out + o;
    const float y0 = tanhf(r[0] + __ldg(&b[o])), sd = 1.f - y0 * y0;
    r[0] = y0;
    r[out] *= sd;
    r[2 * out] *= sd;
    r[3 * out] *= sd;
  }
}

// Output layer after its contraction (H = [P][4][n]): theta = g(h), J_d = g'(h) h_d (Eq. 27),
// the rows (h, h_d) kept for the backward, and the dielectric-set count of the loss.
__global__ void mlp_out_kernel(const float* H, MlpArgs a) {
  const int n = a.out;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.ptot * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gp = e / n;
    const int o = (int)(e % n);
    const float* r = H + gp * 4 * (int64_t)n + o;
    const float h = r[0] + __ldg(&a.b[o]);
    float g0, g1, g2;
    qpk::scale_tanh(a.scale, h, g0, g1, g2);
    reinterpret_cast<float4*>(a.thetaJ)[e] = make_float4(g0, g1 * r[n], g1 * r[2 * n], g1 * r[3 * n]);
    reinterpret_cast<float4*>(a.hout)[e] = make_float4(h, r[n], r[2 * n], r[3 * n]);
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

// Through a hidden layer's tanh, in place on dU = [P][4][in] (cotangents of its outputs y0, y_d)
// with its stored outputs act = [P][4][in]: dH0 = s dU0 - 2 y0 sum_d y_d dU_d, dZ_d = s dU_d.
__global__ void mlp_dact_kernel(float* dU, const float* act, int64_t P, int in) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P * in; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / in;
    const int k = (int)(e % in);
    const int64_t off = p * 4 * (int64_t)in + k;
    const float y0 = act[off], sd = 1.f - y0 * y0;
    const float d1 = dU[off + in], d2 = dU[off + 2 * in], d3 = dU[off + 3 * in];
    const float ys = act[off + in] * d1 + act[off + 2 * in] * d2 + act[off + 3 * in] * d3;
    dU[off] = sd * dU[off] - 2.f * y0 * ys;
    dU[off + in] = sd * d1;
    dU[off + 2 * in] = sd * d2;
    dU[off + 3 * in] = sd * d3;
  }
}

// Bias gradient of one layer per point chunk: slot c gets sum over the chunk's points of the
// value-row cotangent (0 for chunks past the points).
__global__ void mlp_db_kernel(const float* cot, int64_t P, int out, int64_t chunk, int nchunks, float* part,
                              int64_t nW, int64_t b_off) {
  const int c = blockIdx.x;
  for (int o = threadIdx.x; o < out; o += blockDim.x) {
    float acc = 0.f;
    const int64_t p1 = (int64_t)(c + 1) * chunk < P ? (int64_t)(c + 1) * chunk : P;
    for (int64_t p = (int64_t)c * chunk; p < p1; ++p) acc += cot[p * 4 * (int64_t)out + o];
    part[(int64_t)c * nW + b_off + o] = acc;
  }
}

// Zero one parameter segment [off, off + len) of the partial slots c0 .. nchunks - 1.
__global__ void mlp_zero_slots_kernel(float* part, int64_t nW, int64_t off, int64_t len, int c0, int nchunks) {
  const int64_t tot = (int64_t)(nchunks - c0) * len;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
    part[(int64_t)(c0 + e / len) * nW + off + e % len] = 0.f;
}

// Learned period's gradient from the first layer's input cotangents dX = [P][4][2F]:
// sum over points and features of dX . d(features)/dT, added in FP64.
__global__ void mlp_period_kernel(const float* dX, MlpArgs a, double* tgrad) {
  const int in = 2 * a.F;
  float tg = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.ptot * in; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gp = e / in;
    const int k = (int)(e % in);
    int set;
    const float* v = mlp_point(a, gp, set);
    const float4 d = rff_dfeature_dT(a, v, k);
    const float* r = dX + gp * 4 * (int64_t)in + k;
    tg += r[0] * d.x + r[in] * d.y + r[2 * in] * d.z + r[3 * in] * d.w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tg += __shfl_xor_sync(0xffffffffu, tg, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(tgrad, (double)tg);
}

}  // namespace qpm
