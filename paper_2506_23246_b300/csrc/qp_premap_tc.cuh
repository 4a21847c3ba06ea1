// qp_premap_tc.cuh -- the RFF + tanh-MLP premap (F = 64 frequencies, H = 32 units) with its
// first-layer contraction on the 5th-generation tensor cores.
//
// With r = [cos(Omega v), sin(Omega v)] (K = 2F = 128 features) the pre-activation of unit o
// and its x, y, t tangents are h_c[o] = sum_i B[(o, c)][i] r[i], with the first-layer weights
// folded with Omega (d/dv_c turns cos into -sin Omega and sin into cos Omega):
//   B[(o, 0)][i] = W1[o][i],  B[(o, c)][f] = W1[o][F + f] Omega[f][c],  B[(o, c)][F + f] = -W1[o][f] Omega[f][c].
// So the premap forward of a 128-point tile is one [128 points] x [K = 128] x [N = 128
// columns (o, c) = 4 o + c] contraction. Both operands go to the tensor core as FP16 pairs
// (hi + lo of the value times a power of two: 2^12 for |r| <= 1, one scale for B from its
// largest entry), the hi*hi products in one tensor-memory accumulator and the hi*lo + lo*hi
// corrections in a second, added in FP32 by the epilogue.
#pragma once
#include "qp_aux.cuh"
#include "qp_dense.cuh"

namespace qpk {

constexpr int PT_M = 128;                        // points per tile (tensor-memory lanes)
constexpr int PT_THREADS = 256;
constexpr int PT_OPB = PT_M * PG_K * 2;          // one FP16 half of a 128 x 128 operand (4 K blocks of 32)
constexpr int PT_ZMAX = QP_MAXQ;                 // outputs (qubits) the epilogue holds
// The feature operand is built and contracted in two K halves (cos, then sin features) through
// one 64-feature buffer, which the epilogue's output partials reuse: with the folded weights
// resident, two CTAs fit on an SM and one CTA's feature, MMA and epilogue phases run under the
// other's.
struct PtSmem {
  int bh, bl, ah, al, zs, om, b1, w2, b2, ps, bar, total;
};
__host__ __device__ inline PtSmem pt_smem(int n) {
  PtSmem L;
  int o = 0;
  L.bh = o; o += PT_OPB;
  L.bl = o; o += PT_OPB;
  L.ah = o; o += PT_OPB / 2;
  L.al = o; o += PT_OPB / 2;
  L.zs = L.ah;                                   // the second column half's output partials
  L.om = o; o += 3 * PG_F * 4;
  L.b1 = o; o += PG_H * 4;
  L.w2 = o; o += n * PG_H * 4;
  L.b2 = o; o += ((n + 3) & ~3) * 4;
  L.ps = o; o += PT_M * 3 * 4;
  o = (o + 15) & ~15;
  L.bar = o; o += 16;
  L.total = o;
  return L;
}
// Byte offset of FP16 element (row r, feature k) of a 128 x 128 operand: four K blocks of 32,
// each in the K-major core-matrix layout of the other contractions.
__device__ __forceinline__ uint32_t pt_off(int r, int k) {
  return (uint32_t)((k >> 5) * (PT_M * qpd::HKC * 2)) + qpd::core_off_h(r, k & 31);
}

__global__ void __launch_bounds__(PT_THREADS, 2) premap_fwd_tc_kernel(PremapArgs a) {
  extern __shared__ __align__(1024) unsigned char ps_[];
  const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const PtSmem L = pt_smem(n);
  float* om = reinterpret_cast<float*>(ps_ + L.om);
  float* b1 = reinterpret_cast<float*>(ps_ + L.b1);
  float* W2 = reinterpret_cast<float*>(ps_ + L.w2);
  float* b2 = reinterpret_cast<float*>(ps_ + L.b2);
  float* Ps = reinterpret_cast<float*>(ps_ + L.ps);
  float4* Zs = reinterpret_cast<float4*>(ps_ + L.zs);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ps_ + L.bar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(ps_ + L.bar + 8);
  const float* W1 = a.params + 3 * PG_F;
  if (warp == 0) qptc::tmem_alloc(tslot, 256);
  if (tid == 0) qptc::mbar_init(mbar, 1);
  for (int i = tid; i < 3 * PG_F; i += blockDim.x) om[i] = a.params[i];
  for (int i = tid; i < PG_H; i += blockDim.x) b1[i] = W1[PG_H * PG_K + i];
  for (int i = tid; i < n * PG_H; i += blockDim.x) W2[i] = W1[PG_H * PG_K + PG_H + i];
  for (int i = tid; i < n; i += blockDim.x) b2[i] = W1[PG_H * PG_K + PG_H + n * PG_H + i];
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  // the first-layer weights, staged in the (not yet used) feature buffer
  float* W1s = reinterpret_cast<float*>(ps_ + L.ah);
  if ((reinterpret_cast<uintptr_t>(W1) & 15) == 0) {
    for (int i = tid; i < PG_H * PG_K / 4; i += blockDim.x)
      reinterpret_cast<float4*>(W1s)[i] = __ldg(reinterpret_cast<const float4*>(W1) + i);
  } else {   // a parameter vector that is not 16-byte aligned
    for (int i = tid; i < PG_H * PG_K; i += blockDim.x) W1s[i] = __ldg(W1 + i);
  }
  __syncthreads();
  // folded weights: thread -> (column, 8 consecutive features), eight items each
  auto bval = [&](int col, int k) {
    const int o = col >> 2, c = col & 3;
    if (c == 0) return W1s[o * PG_K + k];
    if (k < PG_F) return W1s[o * PG_K + PG_F + k] * om[3 * k + c - 1];
    return -W1s[o * PG_K + (k - PG_F)] * om[3 * (k - PG_F) + c - 1];
  };
  float bmax = 0.f;
  for (int it = tid; it < PG_N * (PG_K / 8); it += blockDim.x) {
    const int col = it & (PG_N - 1), k0 = (it >> 7) * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e) bmax = fmaxf(bmax, fabsf(bval(col, k0 + e)));
  }
  __shared__ float red[PT_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  if (lane == 0) red[warp] = bmax;
  __syncthreads();
  bmax = 0.f;
  for (int w = 0; w < PT_THREADS / 32; ++w) bmax = fmaxf(bmax, red[w]);
  const float sB = qpd::pow2_scale(bmax), sA = qpd::pow2_scale(1.f);
  const float unsc = 1.f / (sA * sB);
  for (int it = tid; it < PG_N * (PG_K / 8); it += blockDim.x) {
    const int col = it & (PG_N - 1), k0 = (it >> 7) * 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = bval(col, k0 + e);
    uint4 h8, l8;
    qpd::pack_h8(v, sB, h8, l8);
    *reinterpret_cast<uint4*>(ps_ + L.bh + pt_off(col, k0)) = h8;
    *reinterpret_cast<uint4*>(ps_ + L.bl + pt_off(col, k0)) = l8;
  }
  const uint32_t id = qptc::idesc(0, PT_M, PG_N);
  const uint32_t t_main = tmem, t_corr = tmem + PG_N;
  // epilogue roles: tensor-memory lane group (warp % 4) = 32 points, column half (warp / 4)
  const int pr = 32 * (warp & 3) + lane, ch = warp >> 2;
  bool ok = true;
  const int64_t ntiles = (a.ptot + PT_M - 1) / PT_M;
  uint32_t phase = 0;   // parity of the next MMA completion (two per tile)
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t p0 = tile * PT_M;
    __syncthreads();   // the previous tile's epilogue is done with the point coordinates
    for (int e = tid; e < PT_M * 3; e += blockDim.x) {
      const int64_t gp = p0 + e / 3;
      float v = 0.f;
      if (gp < a.ptot) {
        int set;
        int64_t li;
        v = point_ptr(a, gp, set, li)[e % 3];
      }
      Ps[e] = v;
    }
    __syncthreads();
    // feature operand in two K halves through one buffer: cos features (K 0..63), then sin
    // features (K 64..127); thread -> (point, 8 consecutive frequencies)
    for (int half = 0; half < 2 && ok; ++half) {
      if (half == 1) {   // the first half's MMAs must be done reading the buffer
        ok = __syncthreads_and(qptc::mbar_wait(mbar, phase));
        phase ^= 1;
        if (!ok) break;
      }
      for (int it = tid; it < PT_M * (PG_F / 8); it += blockDim.x) {
        const int p = it & (PT_M - 1), f0 = (it >> 7) * 8;
        const float x = Ps[3 * p], y = Ps[3 * p + 1], t = Ps[3 * p + 2];
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int f = f0 + e;
          const float ang = om[3 * f] * x + om[3 * f + 1] * y + om[3 * f + 2] * t;
          v[e] = half == 0 ? cosf(ang) : sinf(ang);
        }
        uint4 h8, l8;
        qpd::pack_h8(v, sA, h8, l8);
        *reinterpret_cast<uint4*>(ps_ + L.ah + pt_off(p, f0)) = h8;
        *reinterpret_cast<uint4*>(ps_ + L.al + pt_off(p, f0)) = l8;
      }
      qptc::fence_proxy_async();
      __syncthreads();
      if (tid == 0) {
        qptc::fence_after();
        const uint32_t ah0 = qptc::smem_u32(ps_ + L.ah), al0 = qptc::smem_u32(ps_ + L.al);
        const uint32_t bh0 = qptc::smem_u32(ps_ + L.bh), bl0 = qptc::smem_u32(ps_ + L.bl);
#pragma unroll
        for (int ks = 0; ks < PG_F / 16; ++ks) {
          const uint32_t aoff = (ks >> 1) * (PT_M * qpd::HKC * 2) + (ks & 1) * 256;
          const uint32_t boff = aoff + half * (PT_OPB / 2);   // the B rows' K half
          const uint64_t ah = qptc::desc_kmajor(ah0 + aoff, 128, (qpd::HKC / 8) * 128);
          const uint64_t al = qptc::desc_kmajor(al0 + aoff, 128, (qpd::HKC / 8) * 128);
          const uint64_t bh = qptc::desc_kmajor(bh0 + boff, 128, (qpd::HKC / 8) * 128);
          const uint64_t bl = qptc::desc_kmajor(bl0 + boff, 128, (qpd::HKC / 8) * 128);
          const uint32_t acc = (half > 0 || ks > 0) ? 1u : 0u;
          qptc::mma_f16(t_main, ah, bh, id, acc);
          qptc::mma_f16(t_corr, ah, bl, id, acc);
          qptc::mma_f16(t_corr, al, bh, id, 1u);
        }
        qptc::commit(mbar);
      }
    }
    if (!ok) break;
    ok = __syncthreads_and(qptc::mbar_wait(mbar, phase));
    phase ^= 1;
    if (!ok) break;
    qptc::fence_after();
    // epilogue: this thread's point, units 16 ch .. 16 ch + 15
    const int64_t gp = p0 + pr;
    float4 z[PT_ZMAX];
#pragma unroll
    for (int j = 0; j < PT_ZMAX; ++j) z[j] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int hh = 0; hh < 4; ++hh) {
      float vm[16], vc[16];
      const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
      qptc::tmem_ld16(t_main + lanes + 64 * ch + 16 * hh, vm);
      qptc::tmem_ld16(t_corr + lanes + 64 * ch + 16 * hh, vc);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = 16 * ch + 4 * hh + q;
        const float h0 = (vm[4 * q] + vc[4 * q]) * unsc, h1 = (vm[4 * q + 1] + vc[4 * q + 1]) * unsc;
        const float h2 = (vm[4 * q + 2] + vc[4 * q + 2]) * unsc, h3 = (vm[4 * q + 3] + vc[4 * q + 3]) * unsc;
        const float u = tanhf(h0 + b1[o]);
        const float du = 1.f - u * u;
        const float4 u4 = make_float4(u, du * h1, du * h2, du * h3);
        if (a.u1 && gp < a.ptot) reinterpret_cast<float4*>(a.u1)[gp * PG_H + o] = u4;
#pragma unroll
        for (int j = 0; j < PT_ZMAX; ++j)
          if (j < n) {
            const float w = W2[j * PG_H + o];
            z[j].x += w * u4.x; z[j].y += w * u4.y; z[j].z += w * u4.z; z[j].w += w * u4.w;
          }
      }
    }
    qptc::fence_before();
    if (ch == 1) {
#pragma unroll
      for (int j = 0; j < PT_ZMAX; ++j)
        if (j < n) Zs[pr * PT_ZMAX + j] = z[j];
    }
    __syncthreads();   // also: tensor memory and the feature operand are free for the next tile
    if (ch == 0) {
      if (gp < a.ptot) {
        float4* out = reinterpret_cast<float4*>(a.thetaJ) + gp * n;
#pragma unroll
        for (int j = 0; j < PT_ZMAX; ++j)
          if (j < n) {
            const float4 zo = Zs[pr * PT_ZMAX + j];
            const float z0 = z[j].x + zo.x + b2[j];
            float g0, g1, g2;
            scale_tanh(a.scale, z0, g0, g1, g2);
            out[j] = make_float4(g0, g1 * (z[j].y + zo.y), g1 * (z[j].z + zo.z), g1 * (z[j].w + zo.w));
            if (a.cs) {
              // half-angle factors of the tensor-core path's product states
              float sn, c;
              sincosf(0.5f * g0, &sn, &c);
              a.cs[gp * n + j] = make_float2(c, sn);
            }
          }
      }
      // collocation points inside the dielectric disk, counted once per point
      bool inside = false;
      if (a.medium == 1 && gp < a.npts[0]) {
        const float dx = Ps[3 * pr] - a.disk_x0, dy = Ps[3 * pr + 1] - a.disk_y0;
        inside = __fmaf_rn(dx, dx, dy * dy) < a.disk_r * a.disk_r;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, inside);
      if (lane == 0 && bal) atomicAdd(&a.counts[0], __popc(bal));
    }
  }
  if (!ok && tid == 0) {
    if (a.status) atomicExch(a.status, 6);
    qptc::mbar_wait(mbar, phase ^ 1);  // the last MMAs must finish before tensor memory is freed
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, 256);
}

// ---- premap backward: per 64-point tile the SIMT phases of the FP32 kernel (dL/dz through the
// output layer and the scaling, dL/dh through tanh, the output-layer weight gradient), and the
// first-layer weight gradient D[(o, c)][i] = sum_p d1_p[(o, c)] r_p[i] as one [128 (o, c)] x
// [128 features] x [K = 64 points] tensor-core contraction on FP16 pairs (d1 scaled by one
// power of two per tile, the features by 2^12). Each tile's product comes back from tensor
// memory into FP32 registers, so the sum over tiles is the FP32 sum of the SIMT kernel; the
// Omega fold-back at the end is unchanged.
constexpr int PB_OPB = 128 * PG_TP * 2;   // one FP16 half of a 128-row, K = 64 operand
__host__ __device__ inline int pb_smem(int n) {
  // [A hi, A lo, B hi, B lo] (then the 128 x 129 float result, reaching into Us), Us, Dz,
  // Omega, W2, b2, points, db1 partials, per-warp maxima, mbarrier + tensor-memory slot
  return 4 * PB_OPB + PG_TP * PG_US * 16 + PG_TP * n * 16 + 3 * PG_F * 4 + n * PG_H * 4 + ((n + 3) & ~3) * 4 +
         PG_TP * 3 * 4 + 8 * PG_H * 4 + 8 * 4 + 16;
}
__device__ __forceinline__ uint32_t pb_off(int r, int k) {
  return (uint32_t)((k >> 5) * (128 * qpd::HKC * 2)) + qpd::core_off_h(r, k & 31);
}

__global__ void __launch_bounds__(PG_THREADS, 2) premap_bwd_tc_kernel(PremapArgs a, float* part, int32_t nW) {
  extern __shared__ __align__(1024) unsigned char pb_[];
  const int n = a.n, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* Ah = pb_;
  unsigned char* Al = pb_ + PB_OPB;
  unsigned char* Bh = pb_ + 2 * PB_OPB;
  unsigned char* Bl = pb_ + 3 * PB_OPB;
  float4* Us = reinterpret_cast<float4*>(pb_ + 4 * PB_OPB);   // [TP][PG_US] (u, u_x, u_y, u_t)
  float4* Dz = Us + PG_TP * PG_US;                             // [TP][n] dL/dz (c = 0..3)
  float* om = reinterpret_cast<float*>(Dz + PG_TP * n);        // [F][3]
  float* W2 = om + 3 * PG_F;                                   // [n][H]
  float* b2 = W2 + n * PG_H;
  float* Ps = b2 + ((n + 3) & ~3);                             // [TP][3]
  float* red = Ps + PG_TP * 3;                                 // [8][H] db1 partials
  float* wmax = red + 8 * PG_H;                                // [8] per-warp max |d1|
  uint64_t* mbar = reinterpret_cast<uint64_t*>(wmax + 8);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  float* Dm = reinterpret_cast<float*>(pb_);                   // at the end: [128][129] result
  const float* W1 = a.params + 3 * PG_F;
  if (warp == 0) qptc::tmem_alloc(tslot, 128);
  if (tid == 0) qptc::mbar_init(mbar, 1);
  for (int i = tid; i < 3 * PG_F; i += blockDim.x) om[i] = a.params[i];
  for (int i = tid; i < n * PG_H; i += blockDim.x) W2[i] = W1[PG_H * PG_K + PG_H + i];
  for (int i = tid; i < n; i += blockDim.x) b2[i] = W1[PG_H * PG_K + PG_H + n * PG_H + i];
  qptc::fence_before();
  __syncthreads();   // the fold at the end reads Omega also in blocks without a tile
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = qptc::idesc(0, 128, PG_K);
  const float sB = qpd::pow2_scale(1.f);
  const int ow = tid & 31, pw = tid >> 5;       // (unit, point row) of the dW2 phase
  float acc[64];                                // this thread's row m, 64 columns of D
#pragma unroll
  for (int q = 0; q < 64; ++q) acc[q] = 0.f;
  const int m = 32 * (warp & 3) + lane, chalf = warp >> 2;
  float w2acc[2] = {0.f, 0.f}, b2acc[2] = {0.f, 0.f}, b1acc = 0.f;   // outputs pw, pw + 8
  bool ok = true;
  uint32_t phase = 0;
  const int64_t ntiles = (a.ptot + PG_TP - 1) / PG_TP;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, phase ^= 1) {
    const int64_t p0 = tile * PG_TP;
    __syncthreads();   // every table of the previous tile is consumed
    pg_load_points(a, p0, Ps);
    for (int e = tid; e < PG_TP * PG_H; e += blockDim.x) {
      const int p = e / PG_H, o = e % PG_H;
      const int64_t gp = p0 + p;
      Us[p * PG_US + o] = gp < a.ptot ? reinterpret_cast<const float4*>(a.u1)[gp * PG_H + o]
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    // dL/dz of point tid / 4, outputs j = tid % 4 + 4 jj: theta = g(z_0), J_c = g'(z_0) z_c
    {
      const int p = tid >> 2, j0 = tid & 3;
      const int64_t gp = p0 + p;
      float4 z[3];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) z[jj] = make_float4(j0 + 4 * jj < n ? b2[j0 + 4 * jj] : 0.f, 0.f, 0.f, 0.f);
      for (int o = 0; o < PG_H; ++o) {
        const float4 u4 = Us[p * PG_US + o];
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
          const int j = j0 + 4 * jj;
          if (j < n) {
            const float w = W2[j * PG_H + o];
            z[jj].x += w * u4.x; z[jj].y += w * u4.y; z[jj].z += w * u4.z; z[jj].w += w * u4.w;
          }
        }
      }
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const int j = j0 + 4 * jj;
        if (j < n) {
          float g0, g1, g2;
          scale_tanh(a.scale, z[jj].x, g0, g1, g2);
          const float4 dt = gp < a.ptot ? reinterpret_cast<const float4*>(a.dthetaJ)[gp * n + j]
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
          const float dz0 = dt.x * g1 + g2 * (dt.y * z[jj].y + dt.z * z[jj].z + dt.w * z[jj].w);
          Dz[p * n + j] = make_float4(dz0, dt.y * g1, dt.z * g1, dt.w * g1);
        }
      }
    }
    // feature operand B[i][p] (K = points): thread -> (frequency, 8 consecutive points)
    for (int e = tid; e < PG_F * (PG_TP / 8); e += blockDim.x) {
      const int f = e & (PG_F - 1), pg8 = (e >> 6) * 8;
      float cv[8], sv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int p = pg8 + q;
        sincosf(om[3 * f] * Ps[3 * p] + om[3 * f + 1] * Ps[3 * p + 1] + om[3 * f + 2] * Ps[3 * p + 2], &sv[q], &cv[q]);
      }
      uint4 h8, l8;
      qpd::pack_h8(cv, sB, h8, l8);
      *reinterpret_cast<uint4*>(Bh + pb_off(f, pg8)) = h8;
      *reinterpret_cast<uint4*>(Bl + pb_off(f, pg8)) = l8;
      qpd::pack_h8(sv, sB, h8, l8);
      *reinterpret_cast<uint4*>(Bh + pb_off(PG_F + f, pg8)) = h8;
      *reinterpret_cast<uint4*>(Bl + pb_off(PG_F + f, pg8)) = l8;
    }
    __syncthreads();
    // dW2[j][o] += sum_p dz_j . u_o (c = 0..3), db2[j] += sum_p dz_j0: warp j (and j - 8), lane o
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int j = pw + 8 * jj;
      if (j < n) {
        for (int p = 0; p < PG_TP; ++p) {
          const float4 d = Dz[p * n + j], u4 = Us[p * PG_US + ow];
          w2acc[jj] += d.x * u4.x + d.y * u4.y + d.z * u4.z + d.w * u4.w;
          b2acc[jj] += d.x;
        }
      }
    }
    // dL/du_o = sum_j W2[j][o] dz_j, then through tanh: d1 = dL/dh; thread -> (unit ow, 8
    // consecutive points from 8 pw)
    float d1v[4][8];
    float dm = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int p = 8 * pw + q;
      float4 gu = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int j = 0; j < n; ++j) {
        const float w = W2[j * PG_H + ow];
        const float4 d = Dz[p * n + j];
        gu.x += w * d.x; gu.y += w * d.y; gu.z += w * d.z; gu.w += w * d.w;
      }
      const float4 u4 = Us[p * PG_US + ow];
      const float du = 1.f - u4.x * u4.x;
      const float g0 = gu.x * du - 2.f * u4.x * (gu.y * u4.y + gu.z * u4.z + gu.w * u4.w);
      d1v[0][q] = g0; d1v[1][q] = gu.y * du; d1v[2][q] = gu.z * du; d1v[3][q] = gu.w * du;
      b1acc += g0;
#pragma unroll
      for (int c = 0; c < 4; ++c) dm = fmaxf(dm, fabsf(d1v[c][q]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (lane == 0) wmax[warp] = dm;
    __syncthreads();
    dm = 0.f;
#pragma unroll
    for (int w = 0; w < PG_THREADS / 32; ++w) dm = fmaxf(dm, wmax[w]);
    const float sD = qpd::pow2_scale(dm);
    // d1 operand A[(o, c)][p] (K = points)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint4 h8, l8;
      qpd::pack_h8(d1v[c], sD, h8, l8);
      *reinterpret_cast<uint4*>(Ah + pb_off(4 * ow + c, 8 * pw)) = h8;
      *reinterpret_cast<uint4*>(Al + pb_off(4 * ow + c, 8 * pw)) = l8;
    }
    qptc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      qptc::fence_after();
      const uint32_t ah0 = qptc::smem_u32(Ah), al0 = qptc::smem_u32(Al);
      const uint32_t bh0 = qptc::smem_u32(Bh), bl0 = qptc::smem_u32(Bl);
#pragma unroll
      for (int ks = 0; ks < PG_TP / 16; ++ks) {
        const uint32_t off = (ks >> 1) * (128 * qpd::HKC * 2) + (ks & 1) * 256;
        const uint64_t ah = qptc::desc_kmajor(ah0 + off, 128, (qpd::HKC / 8) * 128);
        const uint64_t al = qptc::desc_kmajor(al0 + off, 128, (qpd::HKC / 8) * 128);
        const uint64_t bh = qptc::desc_kmajor(bh0 + off, 128, (qpd::HKC / 8) * 128);
        const uint64_t bl = qptc::desc_kmajor(bl0 + off, 128, (qpd::HKC / 8) * 128);
        qptc::mma_f16(tmem, ah, bh, id, ks > 0 ? 1u : 0u);
        qptc::mma_f16(tmem, ah, bl, id, 1u);
        qptc::mma_f16(tmem, al, bh, id, 1u);
      }
      qptc::commit(mbar);
    }
    ok = __syncthreads_and(qptc::mbar_wait(mbar, phase));
    if (!ok) break;
    qptc::fence_after();
    {
      const float us = 1.f / (sD * sB);
      const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
      float v[32];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        qptc::tmem_ld32(tmem + lanes + 64 * chalf + 32 * hh, v);
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[32 * hh + q] = fmaf(v[q], us, acc[32 * hh + q]);
      }
    }
    qptc::fence_before();
  }
  if (!ok && tid == 0) {
    if (a.status) atomicExch(a.status, 6);
    qptc::mbar_wait(mbar, phase);   // the tile's MMAs must finish before tensor memory is freed
  }
  __syncthreads();   // the operand buffers are free: the result table takes their place
#pragma unroll
  for (int q = 0; q < 64; ++q) Dm[m * 129 + 64 * chalf + q] = acc[q];
  __syncthreads();
  // fold D back into dW1 (thread: units ty, ty + 16; frequencies f = 4 tx + ii)
  const int ty = tid >> 4, tx = tid & 15;
  float* out = part + (int64_t)blockIdx.x * nW;
#pragma unroll
  for (int uu = 0; uu < 2; ++uu) {
    const int o = ty + 16 * uu;
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int f = tx * 4 + ii;
      const float ox = om[3 * f], oy = om[3 * f + 1], ot = om[3 * f + 2];
      const float* r0 = Dm + (4 * o) * 129;
      const float cosp = r0[f], sinp = r0[PG_F + f];
      const float dwc = cosp - (ox * r0[129 + PG_F + f] + oy * r0[2 * 129 + PG_F + f] + ot * r0[3 * 129 + PG_F + f]);
      const float dws = sinp + (ox * r0[129 + f] + oy * r0[2 * 129 + f] + ot * r0[3 * 129 + f]);
      out[o * PG_K + f] = dwc;
      out[o * PG_K + PG_F + f] = dws;
    }
  }
  red[pw * PG_H + ow] = b1acc;
  __syncthreads();
  if (tid < PG_H) {
    float t = 0.f;
    for (int r = 0; r < PG_THREADS / 32; ++r) t += red[r * PG_H + tid];
    out[PG_H * PG_K + tid] = t;
  }
#pragma unroll
  for (int jj = 0; jj < 2; ++jj) {
    const int j = pw + 8 * jj;
    if (j < n) {
      out[PG_H * PG_K + PG_H + j * PG_H + ow] = w2acc[jj];
      if (ow == 0) out[PG_H * PG_K + PG_H + n * PG_H + j] = b2acc[jj];
    }
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, 128);
  // launched as the programmatic dependent of the gate sweep: finish only after the sweep has,
  // so that the launches after this one see its results (no-op for an ordinary launch)
  qptc::pdl_wait();
}

}  // namespace qpk
