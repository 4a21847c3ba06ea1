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

}  // namespace qpk
