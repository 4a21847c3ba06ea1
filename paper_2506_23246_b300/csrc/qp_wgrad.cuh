// qp_wgrad.cuh -- weight-gradient contraction G = sum over (point, vector) rows of
// R Lambda^H on the tensor cores (3xTF32), FP32 partials per row range.
#pragma once
#include "qp_dense.cuh"

namespace qpd {

// ------------------------------------------------------------------------- weight-gradient GEMM
// G_part[slot][k][o] = sum over the slot's (point, vector) rows of R_s[k] * Lambda_s[o]:
// M = 128 basis indices k, N = min(512, 2^(n+1)) costate components o = (amp, re|im) as one or
// two N = 256 MMAs (all of the row's components in one CTA: R is generated once), K = 16
// (point, vector) rows per step. Steps never straddle point sets: a collocation step holds
// 4 points x 4 vectors (rows consecutive in the costate buffer), an IC/BC step 16 points x 1.
//
// R comes from per-point tables: k = (high bits, 5 low bits); the low five qubits give a
// 32-entry table Lo, the others (bits 5, 6 vary inside a 128-row tile) a 4-entry table H,
// both as a value and its three tangents (forward-mode duals), so each element of R is one
// dual product H[k >> 5] x Lo[k & 31].
//
// Persistent CTAs: CTA b owns tile b % tiles and a balanced range of K-steps; every `fl`
// steps (<= 512 rows, the FP32 accumulation length) the tensor-memory accumulator is flushed
// to its own partial slot, summed later in compensated FP32.
constexpr int WKC = 16;
constexpr int WG_THREADS = 256;

struct WgArgs {
  const float* thetaJ;        // [P][n] float4
  const float2* lam;          // [P][4][dim]
  float* part;                // [nslots][dim][2 dim]
  int32_t n;
  int64_t npts[3], pt_base[3];
  int64_t kc_end[3];          // cumulative 16-row step counts per set
  int32_t tiles, ngroups, spc, fl;  // tiles, CTAs per tile, partial slots per CTA, steps per slot
  int32_t* status;
};

struct WgSmem {
  int a_bytes, b_bytes, stage, fac, lo, hi, bars, total;
};
__host__ __device__ inline WgSmem wg_smem(int n) {
  WgSmem w;
  const int nt = (2 << n) < 512 ? (2 << n) : 512;
  w.a_bytes = TM * WKC * 4;
  w.b_bytes = nt * WKC * 4;
  w.stage = 2 * w.a_bytes + 2 * w.b_bytes;
  int o = 2 * w.stage;
  w.fac = o; o += 2 * 16 * QP_MAXQ * 2 * 16;   // [2][16 pts][q][2] float4
  w.lo = o; o += 16 * 32 * 16;                 // [16 pts][32] float4
  w.hi = o; o += 16 * 4 * 16;                  // [16 pts][4] float4
  w.bars = o; o += 64;
  w.total = o;
  return w;
}
__host__ inline int wg_smem_bytes(int n) { return wg_smem(n).total; }

__device__ __forceinline__ void wg_step_geom(const WgArgs& a, int64_t kc, int& set, int64_t& p0, int& ppc) {
  set = kc < a.kc_end[0] ? 0 : (kc < a.kc_end[1] ? 1 : 2);
  const int64_t ck = kc - (set == 0 ? 0 : a.kc_end[set - 1]);
  ppc = set == 0 ? 4 : 16;
  p0 = ck * ppc;
}

// Costate values of one step for this thread's components o (one per N half) and the raw
// angle entry (theta, J) of the (point, qubit) pair this thread stages.
struct WgLoads {
  float lam[2][WKC];
  float4 tj;
};
__device__ __forceinline__ void wg_load(const WgArgs& a, int64_t kc, int tid, int o0, int nhalf, WgLoads& f) {
  const int n = a.n, dim = 1 << n;
  int set, ppc;
  int64_t p0;
  wg_step_geom(a, kc, set, p0, ppc);
  const int64_t np = a.npts[set];
  const float* lamf = reinterpret_cast<const float*>(a.lam);
  const int64_t row0 = (a.pt_base[set] + p0) * 4;
  const int rstep = set == 0 ? 1 : 4;
  const int nvalid = set == 0 ? (int)((np - p0) * 4 < WKC ? (np - p0) * 4 : WKC)
                              : (int)(np - p0 < WKC ? np - p0 : WKC);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int t = 0; t < WKC; ++t)
      f.lam[h][t] = (h < nhalf && t < nvalid) ? __ldg(lamf + (row0 + (int64_t)t * rstep) * (2 * dim) + o0 + h * 256) : 0.f;
  }
  const int pl = tid / n, q = tid % n;
  f.tj = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid < ppc * n && p0 + pl < np)
    f.tj = __ldg(reinterpret_cast<const float4*>(a.thetaJ) + (a.pt_base[set] + p0 + pl) * n + q);
}

// Per (point, qubit) factors: (cos, sin of theta/2, J_x, J_y), (J_t, valid, ., .).
__device__ __forceinline__ void wg_fac(float4* fac, int tid, int n, int ppc, const float4& tq) {
  if (tid < ppc * n) {
    float sn, cs;
    sincosf(0.5f * tq.x, &sn, &cs);
    fac[tid * 2] = make_float4(cs, sn, tq.y, tq.z);
    fac[tid * 2 + 1] = make_float4(tq.w, 0.f, 0.f, 0.f);
  }
}

// One qubit factor of the product state as a dual (value, d/dx, d/dy, d/dt).
__device__ __forceinline__ float4 wg_dmul(const float4& p, const float4& f0, const float4& f1, bool bit) {
  const float f = bit ? f0.y : f0.x, d = bit ? 0.5f * f0.x : -0.5f * f0.y;
  return make_float4(p.x * f, p.y * f + p.x * d * f0.z, p.z * f + p.x * d * f0.w, p.w * f + p.x * d * f1.x);
}

__global__ void __launch_bounds__(WG_THREADS, 1) dense_wgrad_gemm_kernel(WgArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int n = a.n, dim = 1 << n;
  const WgSmem L = wg_smem(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NT = (2 << n) < 512 ? (2 << n) : 512, nhalf = NT / 256;
  const int tile = blockIdx.x % a.tiles, lb = blockIdx.x / a.tiles;
  const int nmt = dim / TM;
  const int mt = tile % nmt, nt = tile / nmt;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);  // mma_done[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.bars + 32);
  float4* facb = reinterpret_cast<float4*>(sm + L.fac);
  float4* tlo = reinterpret_cast<float4*>(sm + L.lo);
  float4* thi = reinterpret_cast<float4*>(sm + L.hi);
  if (warp == 0) qptc::tmem_alloc(tslot, NT);
  if (tid == 0) { qptc::mbar_init(&bars[0], 1); qptc::mbar_init(&bars[1], 1); }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = qptc::idesc(2, TM, 256);
  const int64_t nkc = a.kc_end[2];
  const int64_t c0 = (int64_t)lb * nkc / a.ngroups, c1 = (int64_t)(lb + 1) * nkc / a.ngroups;
  const int o0 = nt * NT + tid;          // costate components staged by this thread (+256)
  const int kk = tid & (TM - 1), khalf = tid >> 7;
  bool ok = true;
  uint32_t it = 0;
  int64_t last_commit = -1;
  int slot = 0;
  bool fresh = true;                     // next MMA starts a new partial
  WgLoads cur, nxt;
  if (c0 < c1) {
    int set, ppc;
    int64_t p0;
    wg_step_geom(a, c0, set, p0, ppc);
    wg_load(a, c0, tid, o0, nhalf, cur);
    wg_fac(facb + (c0 & 1) * (16 * QP_MAXQ * 2), tid, n, ppc, cur.tj);
    if (c0 + 1 < c1) wg_load(a, c0 + 1, tid, o0, nhalf, nxt);
  }
  __syncthreads();
  // epilogue of one partial: 128 x NT accumulator -> part[slot]; warps w, w + 4 share lanes
  auto flush = [&](int sl, bool zero) {
    const int lrow = (warp & 3) * 32 + lane, chalf = warp >> 2;
    const int ncols = NT / 2;
    float* outp = a.part + (((int64_t)(lb * a.spc + sl) * dim) + mt * TM + lrow) * (2 * dim) + nt * NT + chalf * ncols;
    if (!zero) {
      qptc::fence_after();
      float v[32];
      for (int c = 0; c < ncols; c += 32) {
        qptc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + chalf * ncols + c, v);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          reinterpret_cast<float4*>(outp + c)[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
      }
    } else {
      for (int c = 0; c < ncols; c += 4) *reinterpret_cast<float4*>(outp + c) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    qptc::fence_before();
  };
  for (int64_t kc = c0; kc < c1 && ok; ++kc, ++it) {
    const uint32_t st = it & 1;
    unsigned char* sA = sm + st * L.stage;
    unsigned char* sB = sA + 2 * L.a_bytes;
    int set, ppc;
    int64_t p0;
    wg_step_geom(a, kc, set, p0, ppc);
    bool w_ok = true;
    if (it >= 2) w_ok = qptc::mbar_wait(&bars[st], ((it - 2) >> 1) & 1);
    ok = __syncthreads_and(w_ok);   // also orders the previous step's reads of the tables
    if (!ok) break;
    const float4* fac = facb + (kc & 1) * (16 * QP_MAXQ * 2);
    // tables of this step: Lo over the five low qubits, H over the others for k >> 5 in tile
    for (int idx = tid; idx < ppc * 32; idx += WG_THREADS) {
      const int pl = idx >> 5, e = idx & 31;
      float4 p = make_float4(1.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int b = 4; b >= 0; --b) {
        const int q = n - 1 - b;
        p = wg_dmul(p, fac[(pl * n + q) * 2], fac[(pl * n + q) * 2 + 1], (e >> b) & 1);
      }
      tlo[idx] = p;
    }
    for (int idx = tid; idx < ppc * 4; idx += WG_THREADS) {
      const int pl = idx >> 2, j = idx & 3;
      const int kb = mt * TM + j * 32;
      float4 p = make_float4(1.f, 0.f, 0.f, 0.f);
      for (int q = 0; q < n - 5; ++q)
        p = wg_dmul(p, fac[(pl * n + q) * 2], fac[(pl * n + q) * 2 + 1], (kb >> (n - 1 - q)) & 1);
      thi[idx] = p;
    }
    // factors of the next step (other buffer) and B staging of this step
    if (kc + 1 < c1) {
      int set1, ppc1;
      int64_t p01;
      wg_step_geom(a, kc + 1, set1, p01, ppc1);
      wg_fac(facb + ((kc + 1) & 1) * (16 * QP_MAXQ * 2), tid, n, ppc1, nxt.tj);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h < nhalf) {
        float* Bhi = reinterpret_cast<float*>(sB + h * 2 * (256 * WKC * 4));
        float* Blo = Bhi + 256 * WKC;
#pragma unroll
        for (int g4 = 0; g4 < WKC / 4; ++g4) {
          float4 h4, l4;
          qptc::split_tf32(cur.lam[h][4 * g4], h4.x, l4.x);
          qptc::split_tf32(cur.lam[h][4 * g4 + 1], h4.y, l4.y);
          qptc::split_tf32(cur.lam[h][4 * g4 + 2], h4.z, l4.z);
          qptc::split_tf32(cur.lam[h][4 * g4 + 3], h4.w, l4.w);
          const uint32_t off = core_off16(tid, g4 * 4) / 4;
          *reinterpret_cast<float4*>(Bhi + off) = h4;
          *reinterpret_cast<float4*>(Blo + off) = l4;
        }
      }
    }
    // global loads two steps ahead are in flight while this step is generated and multiplied
    cur = nxt;
    if (kc + 2 < c1) wg_load(a, kc + 2, tid, o0, nhalf, nxt);
    __syncthreads();  // tables visible
    {
      float av[8];
      const int j = kk >> 5, e = kk & 31;
      if (set == 0) {
#pragma unroll
        for (int pi = 0; pi < 2; ++pi) {
          const int pl = khalf * 2 + pi;
          const float4 h = thi[pl * 4 + j], l = tlo[pl * 32 + e];
          av[4 * pi] = h.x * l.x;
          av[4 * pi + 1] = h.y * l.x + h.x * l.y;
          av[4 * pi + 2] = h.z * l.x + h.x * l.z;
          av[4 * pi + 3] = h.w * l.x + h.x * l.w;
        }
      } else {
#pragma unroll
        for (int pi = 0; pi < 8; ++pi) {
          const int pl = khalf * 8 + pi;
          av[pi] = thi[pl * 4 + j].x * tlo[pl * 32 + e].x;
        }
      }
      float* Ahi = reinterpret_cast<float*>(sA);
      float* Alo = reinterpret_cast<float*>(sA + L.a_bytes);
#pragma unroll
      for (int g4 = 0; g4 < 2; ++g4) {
        float4 h4, l4;
        qptc::split_tf32(av[4 * g4], h4.x, l4.x);
        qptc::split_tf32(av[4 * g4 + 1], h4.y, l4.y);
        qptc::split_tf32(av[4 * g4 + 2], h4.z, l4.z);
        qptc::split_tf32(av[4 * g4 + 3], h4.w, l4.w);
        const uint32_t off = core_off16(kk, khalf * 8 + g4 * 4) / 4;
        *reinterpret_cast<float4*>(Ahi + off) = h4;
        *reinterpret_cast<float4*>(Alo + off) = l4;
      }
    }
    qptc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      qptc::fence_after();
      const uint32_t sa = qptc::smem_u32(sA), sb = qptc::smem_u32(sB);
      const uint32_t bblk = 256 * WKC * 4;
#pragma unroll
      for (int ks = 0; ks < WKC / 8; ++ks) {
        const uint64_t ah = qptc::desc_kmajor(sa + ks * 256, 128, (WKC / 4) * 128);
        const uint64_t al = qptc::desc_kmajor(sa + L.a_bytes + ks * 256, 128, (WKC / 4) * 128);
        for (int h = 0; h < nhalf; ++h) {
          const uint64_t bh = qptc::desc_kmajor(sb + h * 2 * bblk + ks * 256, 128, (WKC / 4) * 128);
          const uint64_t bl = qptc::desc_kmajor(sb + h * 2 * bblk + bblk + ks * 256, 128, (WKC / 4) * 128);
          const uint32_t dt = tmem + h * 256;
          qptc::mma_tf32(dt, ah, bh, id, (fresh && ks == 0) ? 0u : 1u);
          qptc::mma_tf32(dt, ah, bl, id, 1u);
          qptc::mma_tf32(dt, al, bh, id, 1u);
        }
      }
      qptc::commit(&bars[st]);
      last_commit = it;
    }
    fresh = false;
    if ((kc - c0 + 1) % a.fl == 0 || kc + 1 == c1) {
      ok = __syncthreads_and(qptc::mbar_wait(&bars[st], (it >> 1) & 1));
      if (!ok) break;
      flush(slot, false);
      ++slot;
      fresh = true;
      __syncthreads();
    }
  }
  if (ok) {
    for (int sl = slot; sl < a.spc; ++sl) flush(sl, true);
  } else {
    if (tid == 0) {
      atomicExch(a.status, 6);
      if (last_commit >= 0) qptc::mbar_wait(&bars[last_commit & 1], ((uint32_t)last_commit >> 1) & 1);
    }
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, NT);
}

}  // namespace qpd
