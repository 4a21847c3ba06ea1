// qp_wgrad.cuh -- weight-gradient contraction G = sum over (point, vector) rows of
// R Lambda^H on the tensor cores (FP16 or TF32 operand pairs), FP32 partials per row range.
#pragma once
#include "qp_dense.cuh"

namespace qpd {

// ------------------------------------------------------------------------- weight-gradient GEMM
// G_part[slot][k][o] = sum over the slot's (point, vector) rows of R_s[k] * Lambda_s[o]. A CTA
// tile covers MTC = min(256, 2^n) basis indices k (one or two M = 128 MMAs) x 256 costate
// components o = (amp, re|im) (N = 256), so tensor memory holds the whole tile (<= 512
// columns) and every costate element is read by one CTA only. K = 16 (point, vector) rows per
// step; steps never straddle point sets: a collocation step holds 4 points x 4 vectors (rows
// consecutive in the costate buffer), an IC/BC step 16 points x 1 vector.
//
// R comes from per-point tables: k = (high bits, 5 low bits); the five low qubits give a
// 32-entry table Lo, the others an 8-entry table H over the bits 5-7 of k inside the tile
// (higher bits fixed by the tile), both as a value and its three tangents (forward-mode
// duals), so each element of R is one dual product H[k >> 5] x Lo[k & 31].
//
// Persistent CTAs: the tiles' steps are laid out tile-major as one sequence (step x = tile *
// nkc + kc) and split into gridDim.x balanced ranges, so every SM gets the same number of steps
// whatever the tile count; a range meets at most two tiles (two segments). Every `fl` steps of
// a segment (<= 512 rows, the FP32 accumulation length in tensor memory), and at its end, the
// accumulator is added into the CTA's partial slot of that tile (a few FP32 adds per element,
// the slot stays in L2); a tile's slot j belongs to the j-th CTA whose range meets the tile,
// and the slots of a tile are summed later in compensated FP32.
//
// Pipeline: the costate rows arrive in a 4-slot shared-memory ring by bulk copies issued three
// steps ahead by a control thread, which also issues the MMAs in step order. The staging is
// done by crews of eight warps, each taking every NC-th step whole (see below).
constexpr int WKC = 16;

// Fire-and-forget vector add into global memory (performed at L2).
__device__ __forceinline__ void red_add_f4(float4* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
constexpr int WG_RING = 4;

// The range of the tile-major step sequence (T steps, G ranges) that holds step x.
__host__ __device__ inline int64_t wg_range_start(int64_t b, int64_t T, int64_t G) { return b * T / G; }
__host__ __device__ inline int64_t wg_cta_of(int64_t x, int64_t T, int64_t G) {
  int64_t b = x * G / T;
  while (b + 1 < G && wg_range_start(b + 1, T, G) <= x) ++b;
  while (b > 0 && wg_range_start(b, T, G) > x) --b;
  return b;
}

struct WgArgs {
  const float* thetaJ;        // [P][n] float4 (theta, J_x, J_y, J_t)
  const float2* cs;           // [P][n] (cos, sin) of theta / 2
  const float* lam;           // costate rows: blocked [2 dim / 256][rtot][256] or rows [P][4][2 dim]
  int64_t rtot;               // rows of the blocked layout (0: row layout)
  float* part;                // [nslots][dim][2 dim]: slot j of a tile is the j-th CTA meeting it
  int32_t n;
  int64_t npts[3], pt_base[3];
  int64_t kc_end[3];          // cumulative 16-row step counts per set
  int32_t tiles, nslots, fl;   // tiles, partial slots per tile, steps per flush
  int32_t* status;
  const int32_t* scal;        // FP16 operands: [2] float bits, bound of |R|, max |lambda|
};

// Byte offset of 16-bit element (row r, K index k) in a K-major WKC-wide block (core matrices
// of 8 rows x 8 elements, K-adjacent ones 128 bytes apart, 8-row groups 256 bytes apart).
__host__ __device__ inline uint32_t core_off_w16(int r, int k) {
  return (uint32_t)((r >> 3) * (WKC / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}


constexpr int WG_TAB4 = 16 * 32 + 16 * 8;                 // Lo [16 pts][32], H [16 pts][8] float4
constexpr int WG_FAC4 = 16 * QP_MAXQ * 2;                 // [16 pts][q][2] float4
__host__ __device__ inline int wg_mtc(int n) { return (1 << n) < 256 ? (1 << n) : 256; }

__device__ __forceinline__ void wg_step_geom(const WgArgs& a, int64_t kc, int& set, int64_t& p0, int& ppc,
                                             int& nvalid) {
  set = kc < a.kc_end[0] ? 0 : (kc < a.kc_end[1] ? 1 : 2);
  const int64_t ck = kc - (set == 0 ? 0 : a.kc_end[set - 1]);
  ppc = set == 0 ? 4 : 16;
  p0 = ck * ppc;
  const int64_t left = (a.npts[set] - p0) * (set == 0 ? 4 : 1);
  nvalid = (int)(left < WKC ? left : WKC);
}

// Angle entry of the (point, qubit) pair `tid` of step kc: (cos, sin of theta/2, J_x, J_y), J_t.
struct WgAng {
  float4 f0;
  float jt;
};
__device__ __forceinline__ WgAng wg_load_ang(const WgArgs& a, int64_t kc, int tid, int n) {
  int set, ppc, nv;
  int64_t p0;
  wg_step_geom(a, kc, set, p0, ppc, nv);
  const int pl = tid / n, q = tid % n;
  WgAng r;
  r.f0 = make_float4(0.f, 0.f, 0.f, 0.f);
  r.jt = 0.f;
  if (tid < ppc * n && p0 + pl < a.npts[set]) {
    const int64_t i = (a.pt_base[set] + p0 + pl) * n + q;
    const float4 tq = __ldg(reinterpret_cast<const float4*>(a.thetaJ) + i);
    const float2 c = __ldg(a.cs + i);
    r.f0 = make_float4(c.x, c.y, tq.y, tq.z);
    r.jt = tq.w;
  }
  return r;
}

// Per (point, qubit) factors: (cos, sin of theta/2, J_x, J_y), (J_t, ., ., .).
__device__ __forceinline__ void wg_fac(float4* fac, int tid, int n, int ppc, const WgAng& g) {
  if (tid < ppc * n) {
    fac[tid * 2] = g.f0;
    fac[tid * 2 + 1] = make_float4(g.jt, 0.f, 0.f, 0.f);
  }
}

// One qubit factor of the product state as a dual (value, d/dx, d/dy, d/dt).
__device__ __forceinline__ float4 wg_dmul(const float4& p, const float4& f0, const float4& f1, bool bit) {
  const float f = bit ? f0.y : f0.x, d = bit ? 0.5f * f0.x : -0.5f * f0.y;
  return make_float4(p.x * f, p.y * f + p.x * d * f0.z, p.z * f + p.x * d * f0.w, p.w * f + p.x * d * f1.x);
}

// Bulk copies of the valid costate rows of step kc (this tile's 256 columns) into `raw`.
__device__ __forceinline__ void wg_copy_rows(const WgArgs& a, int64_t kc, int ntile, float* raw, uint64_t* bar) {
  const int dim = 1 << a.n;
  int set, ppc, nv;
  int64_t p0;
  wg_step_geom(a, kc, set, p0, ppc, nv);
  const uint32_t rowb = 256 * 4;
  qptc::mbar_arrive_expect_tx(bar, nv * rowb);
  const float* lamf = a.lam;
  const int64_t row0 = (a.pt_base[set] + p0) * 4;
  if (a.rtot > 0) {
    // blocked layout: the step's rows are consecutive in every 256-column block
    const int64_t r0 = lam_row(set, p0, 0, a.npts[0], a.pt_base[set]);
    qptc::bulk_g2s(raw, lamf + ((int64_t)ntile * a.rtot + r0) * 256, nv * rowb, bar);
  } else if (set == 0 && 2 * dim == 256) {
    qptc::bulk_g2s(raw, lamf + row0 * (2 * dim), nv * rowb, bar);
  } else {
    const int rstep = set == 0 ? 1 : 4;
    for (int t = 0; t < nv; ++t)
      qptc::bulk_g2s(raw + t * 256, lamf + (row0 + (int64_t)t * rstep) * (2 * dim) + ntile * 256, rowb, bar);
  }
}

// ------------------------------------------------------------------------- crews
// Staging by crews instead of roles: crew c (eight
// warps) takes every NC-th 16-row step and does all of a step's staging work itself -- angle
// factors, R tables, both M sub-tiles of the A operand and the B operand -- into its own
// operand stage c, so NC steps are staged at once and the latency chain of one step (factor
// and table barriers, the dependent dual products, the operand splits) overlaps the chains of
// the other crews instead of setting the pace. A producer warp streams the costate rows into
// the 4-slot ring as soon as a slot is read (up to four steps ahead, never held up by the MMA
// issue); the control warp issues the MMAs in step order; the crew holding a chunk's last step
// drains the accumulator into the CTA's partial slot while the other crews stage the next steps.
constexpr int WGC_CREW = 256;   // threads of a crew
__host__ __device__ constexpr int wgc_ncrew(bool h16) { return h16 ? 3 : 2; }
// crews, then the control warp (MMAs) and the producer warp (costate copies)
__host__ __device__ constexpr int wgc_threads(bool h16) { return wgc_ncrew(h16) * WGC_CREW + 64; }

struct WgcSmem {
  int a_bytes, b_bytes, stage, raw, fac, tab, bars, total;
};
// FP16 pairs: three crews (stages of 32 KiB); TF32 pairs: two (stages of 64 KiB).
__host__ __device__ inline WgcSmem wgc_smem(int n, bool h16) {
  const int esz = h16 ? 2 : 4, nc = wgc_ncrew(h16);
  WgcSmem w;
  w.a_bytes = (wg_mtc(n) / TM) * 2 * TM * WKC * esz;
  w.b_bytes = 2 * 256 * WKC * esz;
  w.stage = w.a_bytes + w.b_bytes;
  int o = nc * w.stage;
  w.raw = o; o += WG_RING * WKC * 256 * 4;
  w.fac = o; o += nc * WG_FAC4 * 16;
  w.tab = o; o += nc * WG_TAB4 * 16;
  // mma_done[3], stage_full[3], raw_full[4], raw_free[4], acc_free, tmem slot
  w.bars = o; o += 256;
  w.total = o;
  return w;
}

// Tables of one step over one crew: Lo entries on the first threads, H entries from the crew's
// second half (a collocation step: Lo on warps 0-3, H on warp 4).
__device__ __forceinline__ void wgc_tables(const float4* fac, float4* tab, int t, int n, int ppc, int kbase,
                                           int nj) {
  float4* tlo = tab;
  float4* thi = tab + 16 * 32;
  for (int idx = t; idx < ppc * 32; idx += WGC_CREW) {
    const int pl = idx >> 5, e = idx & 31;
    float4 p = make_float4(1.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int b = 4; b >= 0; --b) {
      const int q = n - 1 - b;
      p = wg_dmul(p, fac[(pl * n + q) * 2], fac[(pl * n + q) * 2 + 1], (e >> b) & 1);
    }
    tlo[idx] = p;
  }
  for (int idx = (t + WGC_CREW / 2) & (WGC_CREW - 1); idx < ppc * 8; idx += WGC_CREW) {
    const int pl = idx >> 3, j = idx & 7;
    if (j < nj) {
      const int kb = kbase + j * 32;
      float4 p = make_float4(1.f, 0.f, 0.f, 0.f);
      for (int q = 0; q < n - 5; ++q)
        p = wg_dmul(p, fac[(pl * n + q) * 2], fac[(pl * n + q) * 2 + 1], (kb >> (n - 1 - q)) & 1);
      thi[idx] = p;
    }
  }
}

template <bool H16, int NQ>
__global__ void __launch_bounds__(wgc_threads(H16), 1) dense_wgrad_gemm_kernel(WgArgs a) {
  static_assert(NQ >= 7 && NQ <= 10, "weight-gradient contraction: 7 to 10 qubits");
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int n = NQ, dim = 1 << n;
  constexpr int NC = wgc_ncrew(H16);
  constexpr int ESZ = H16 ? 2 : 4;
  const WgcSmem L = wgc_smem(n, H16);
  float sR = 1.f, sL = 1.f;
  if (H16) {
    sR = pow2_scale(__int_as_float(__ldg(a.scal)));
    sL = pow2_scale(__int_as_float(__ldg(a.scal + 1)));
  }
  const float unsc = 1.f / (sR * sL);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool ctrl = warp == NC * 8, prod = warp == NC * 8 + 1;
  const int MTC = wg_mtc(n), msub = MTC / TM, nj = MTC / 32;
  const int nmt = dim / MTC;
  // this CTA's range of the tile-major step sequence: steps v < vb in tile t0 (from its step
  // kc00 on, slot slot0), the rest in tile t0 + 1 (from its first step: slot 0)
  const int64_t nkc = a.kc_end[2];
  const int64_t T = (int64_t)a.tiles * nkc, G = gridDim.x;
  // range of this CTA: where the CTAs divide evenly over the tiles, neighbouring CTAs take
  // different tiles (CTA b: tile b mod tiles)
  const int64_t rb = G % a.tiles == 0 ? (int64_t)(blockIdx.x % a.tiles) * (G / a.tiles) + blockIdx.x / a.tiles
                                      : (int64_t)blockIdx.x;
  // (the host keeps tiles x steps below 2^31, so step counts are 32-bit)
  const int64_t X0 = T > 0 ? wg_range_start(rb, T, G) : 0;
  const int V = T > 0 ? (int)(wg_range_start(rb + 1, T, G) - X0) : 0;
  const int t0 = V > 0 ? (int)(X0 / nkc) : 0;
  const int kc00 = (int)(X0 - (int64_t)t0 * nkc);
  const int vb = (int)nkc - kc00 < V ? (int)nkc - kc00 : V;
  const int slot0 = V > 0 ? (int)(rb - wg_cta_of((int64_t)t0 * nkc, T, G)) : 0;
  // step v: tile, step index in the tile, position and length of its segment, slot
  // (for n <= 8 the host makes the grid a multiple of the tile count: every range then lies
  // inside one tile, and the second segment is compiled out)
  auto step_of = [&](int v, int& tile, int& kc, int& vs, int& slen, int& slot) {
    const bool s1 = NQ >= 9 && v >= vb;
    tile = t0 + (s1 ? 1 : 0);
    kc = s1 ? v - vb : kc00 + v;
    vs = s1 ? v - vb : v;
    slen = s1 ? V - vb : vb;
    slot = s1 ? 0 : slot0;
  };
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* mma_done = bars;          // [NC] MMAs of a crew's stage finished (commit)
  uint64_t* stage_full = bars + 3;    // [NC] a crew's operands written (its 8 warps)
  uint64_t* raw_full = bars + 6;      // [4]  costate rows of a ring slot landed
  uint64_t* raw_free = bars + 10;     // [4]  ring slot read (the 8 warps of the step's crew)
  uint64_t* acc_free = bars + 14;     // accumulator drained (the 8 warps of the draining crew)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.bars + 128);
  float* raw = reinterpret_cast<float*>(sm + L.raw);
  const uint32_t tcols = msub * 256;
  if (warp == 0) qptc::tmem_alloc(tslot, tcols);
  if (tid == 0) {
    for (int i = 0; i < NC; ++i) qptc::mbar_init(&mma_done[i], 1);
    for (int i = 0; i < NC; ++i) qptc::mbar_init(&stage_full[i], 8);
    for (int i = 0; i < WG_RING; ++i) qptc::mbar_init(&raw_full[i], 1);
    for (int i = 0; i < WG_RING; ++i) qptc::mbar_init(&raw_free[i], 8);
    qptc::mbar_init(acc_free, 8);
  }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  // chunk boundaries staggered over the CTAs (a segment's first chunk is shorter by 0 .. 7
  // eighths), so that the drains into L2 do not all fall at the same time
  const int choff = (int)(blockIdx.x & 7) * a.fl / 8;
  bool ok = true;
  if (prod) {
    // ---- producer thread: the costate rows of every step into the ring, once the slot's
    // previous step has been read
    if (lane == 0) {
      int last_copy = -1;
      for (int j = 0; j < V && ok; ++j) {
        if (j >= WG_RING) ok = qptc::mbar_wait(&raw_free[j % WG_RING], (uint32_t)((j - WG_RING) / WG_RING) & 1);
        if (!ok) break;
        int tile, slot, kc, vs, slen;
        step_of(j, tile, kc, vs, slen, slot);
        qptc::fence_proxy_async();
        wg_copy_rows(a, kc, tile / nmt, raw + (j % WG_RING) * (WKC * 256), &raw_full[j % WG_RING]);
        last_copy = j;
      }
      if (!ok) {
        atomicExch(a.status, 6);
        // let the copies in flight land before exiting
        for (int j = last_copy - (WG_RING - 1) < 0 ? 0 : last_copy - (WG_RING - 1); j <= last_copy; ++j)
          qptc::mbar_wait(&raw_full[j % WG_RING], (uint32_t)(j / WG_RING) & 1);
      }
    }
  } else if (ctrl) {
    // ---- control thread: MMAs in step order
    if (lane == 0) {
      int64_t last_commit = -1;
      const uint32_t id = qptc::idesc(H16 ? 0 : 2, TM, 256);
      bool fresh = true;
      int chunk = 0;
      uint32_t it = 0;
      for (int v = 0; v < V && ok; ++v, ++it) {
        const uint32_t c = it % NC, lc = it / NC;
        int tile, slot, kc, vs, slen;
        step_of(v, tile, kc, vs, slen, slot);
        if (fresh && chunk > 0) ok = qptc::mbar_wait(acc_free, (uint32_t)(chunk - 1) & 1);
        if (!ok) break;
        ok = qptc::mbar_wait(&stage_full[c], lc & 1);
        if (!ok) break;
        qptc::fence_after();
        const uint32_t sa = qptc::smem_u32(sm + c * L.stage), sb = sa + L.a_bytes;
        if (H16) {
          const uint32_t ablk = TM * WKC * 2, bblk = 256 * WKC * 2;
          const uint64_t bh = qptc::desc_kmajor(sb, 128, (WKC / 8) * 128);
          const uint64_t bl = qptc::desc_kmajor(sb + bblk, 128, (WKC / 8) * 128);
          for (int u = 0; u < msub; ++u) {
            const uint64_t ah = qptc::desc_kmajor(sa + u * 2 * ablk, 128, (WKC / 8) * 128);
            const uint64_t al = qptc::desc_kmajor(sa + u * 2 * ablk + ablk, 128, (WKC / 8) * 128);
            const uint32_t dt = tmem + u * 256;
            qptc::mma_f16(dt, ah, bh, id, fresh ? 0u : 1u);
            qptc::mma_f16(dt, ah, bl, id, 1u);
            qptc::mma_f16(dt, al, bh, id, 1u);
          }
        }
        const uint32_t ablk = TM * WKC * 4, bblk = 256 * WKC * 4;
#pragma unroll
        for (int ks = 0; ks < (H16 ? 0 : WKC / 8); ++ks) {
          const uint64_t bh = qptc::desc_kmajor(sb + ks * 256, 128, (WKC / 4) * 128);
          const uint64_t bl = qptc::desc_kmajor(sb + bblk + ks * 256, 128, (WKC / 4) * 128);
          for (int u = 0; u < msub; ++u) {
            const uint64_t ah = qptc::desc_kmajor(sa + u * 2 * ablk + ks * 256, 128, (WKC / 4) * 128);
            const uint64_t al = qptc::desc_kmajor(sa + u * 2 * ablk + ablk + ks * 256, 128, (WKC / 4) * 128);
            const uint32_t dt = tmem + u * 256;
            qptc::mma_tf32(dt, ah, bh, id, (fresh && ks == 0) ? 0u : 1u);
            qptc::mma_tf32(dt, ah, bl, id, 1u);
            qptc::mma_tf32(dt, al, bh, id, 1u);
          }
        }
        qptc::commit(&mma_done[c]);
        last_commit = it;
        fresh = false;
        if ((vs + 1 + choff) % a.fl == 0 || vs + 1 == slen) {
          fresh = true;
          ++chunk;
        }
      }
      if (!ok) {
        atomicExch(a.status, 6);
        // let every tensor-core operation of this CTA land before exiting
        if (last_commit >= 0)
          qptc::mbar_wait(&mma_done[last_commit % NC], ((uint32_t)last_commit / NC) & 1);
      }
    }
  } else {
    // ---- crews
    const int crew = warp >> 3, cw = warp & 7, ct = tid - crew * WGC_CREW;
    const int bar_id = 1 + crew;
    float4* fac = reinterpret_cast<float4*>(sm + L.fac) + crew * WG_FAC4;
    float4* tab = reinterpret_cast<float4*>(sm + L.tab) + crew * WG_TAB4;
    unsigned char* sA = sm + crew * L.stage;
    unsigned char* sB = sA + L.a_bytes;
    // drain of the accumulator by this crew: lane quarter cw & 3, half cw >> 2 of the columns
    auto flush = [&](bool add, bool zero, int slot, int tile) {
      const int g = cw & 3, h = cw >> 2;
      const int u = msub == 2 ? h : 0;
      const int cbeg = msub == 2 ? 0 : h * 128, ncols = msub == 2 ? 256 : 128;
      const int64_t krow = (int64_t)(tile % nmt) * MTC + u * TM + g * 32 + lane;
      float* outp = a.part + (((int64_t)slot * dim) + krow) * (2 * dim) + (tile / nmt) * 256 + cbeg;
      if (!zero) {
        float v[32];
        for (int c = 0; c < ncols; c += 32) {
          qptc::tmem_ld32(tmem + ((uint32_t)(g * 32) << 16) + u * 256 + cbeg + c, v);
          float4* o4 = reinterpret_cast<float4*>(outp + c);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float4 r = make_float4(unsc * v[4 * e], unsc * v[4 * e + 1], unsc * v[4 * e + 2], unsc * v[4 * e + 3]);
            if (add) red_add_f4(o4 + e, r);
            else o4[e] = r;
          }
        }
      } else {
        for (int c = 0; c < ncols; c += 4) *reinterpret_cast<float4*>(outp + c) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    // the slots no CTA writes of each tile whose first step this CTA holds: zero, so that the
    // slot sum can take the same slot count for every tile
    if (NQ >= 9 && crew == 0 && V > 0) {
      for (int sg = 0; sg < 2; ++sg) {
        if (sg == 1 && V <= vb) break;
        if (sg == 0 && slot0 != 0) continue;
        const int tz = t0 + sg;
        const int64_t nmeet = wg_cta_of((int64_t)(tz + 1) * nkc - 1, T, G) - rb + 1;
        for (int j = (int)nmeet; j < a.nslots; ++j) flush(false, true, j, tz);
      }
    }
    WgAng g{};
    int tile = 0, slot = 0, kc = 0, vs = 0, slen = 0;
    if (crew < V) {
      step_of(crew, tile, kc, vs, slen, slot);
      g = wg_load_ang(a, kc, ct, n);
    }
    uint32_t cnt = 0;
    for (int v = crew; v < V; v += NC, ++cnt) {
      const uint32_t it = (uint32_t)v;
      step_of(v, tile, kc, vs, slen, slot);
      const int kbase = (tile % nmt) * MTC;
      int set, ppc, nvalid;
      int64_t p0;
      wg_step_geom(a, kc, set, p0, ppc, nvalid);
      // factors of this step, then the angles of the crew's next step
      wg_fac(fac, ct, n, ppc, g);
      if (v + NC < V) {
        int tn, sn, kn, vn, ln;
        step_of(v + NC, tn, kn, vn, ln, sn);
        g = wg_load_ang(a, kn, ct, n);
      }
      ok = qptc::bar_and(bar_id, WGC_CREW, ok);
      if (!ok) break;
      wgc_tables(fac, tab, ct, n, ppc, kbase, nj);
      ok = qptc::bar_and(bar_id, WGC_CREW, ok);
      if (!ok) break;
      bool good = true;
      // the stage is free once the MMAs of the crew's previous step finished
      if (cnt >= 1) good = qptc::mbar_wait(&mma_done[crew], (cnt - 1) & 1);
      // A operand: thread -> basis index k = kbase + ct (both M sub-tiles), all 16 rows
      if (ct < MTC) {
        const int u = ct >> 7, kk = ct & (TM - 1), e = ct & 31, j = ct >> 5;
        const float4* tlo = tab;
        const float4* thi = tab + 16 * 32;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float av[8];
          if (set == 0) {
#pragma unroll
            for (int pi = 0; pi < 2; ++pi) {
              const int pl = h * 2 + pi;
              const float4 hv = thi[pl * 8 + j], l = tlo[pl * 32 + e];
              av[4 * pi] = hv.x * l.x;
              av[4 * pi + 1] = hv.y * l.x + hv.x * l.y;
              av[4 * pi + 2] = hv.z * l.x + hv.x * l.z;
              av[4 * pi + 3] = hv.w * l.x + hv.x * l.w;
            }
          } else {
#pragma unroll
            for (int pi = 0; pi < 8; ++pi) {
              const int pl = h * 8 + pi;
              av[pi] = thi[pl * 8 + j].x * tlo[pl * 32 + e].x;
            }
          }
          if (good) {
            if (H16) {
              uint4 h8, l8;
              pack_h8(av, sR, h8, l8);
              unsigned char* Ab = sA + u * 2 * (TM * WKC * 2);
              const uint32_t off = core_off_w16(kk, h * 8);
              *reinterpret_cast<uint4*>(Ab + off) = h8;
              *reinterpret_cast<uint4*>(Ab + TM * WKC * 2 + off) = l8;
            } else {
              float* Ahi = reinterpret_cast<float*>(sA + u * 2 * (TM * WKC * 4));
              float* Alo = Ahi + TM * WKC;
#pragma unroll
              for (int g4 = 0; g4 < 2; ++g4) {
                float4 h4, l4;
                qptc::split_tf32_fast(av[4 * g4], h4.x, l4.x);
                qptc::split_tf32_fast(av[4 * g4 + 1], h4.y, l4.y);
                qptc::split_tf32_fast(av[4 * g4 + 2], h4.z, l4.z);
                qptc::split_tf32_fast(av[4 * g4 + 3], h4.w, l4.w);
                const uint32_t off = core_off16(kk, h * 8 + g4 * 4) / 4;
                *reinterpret_cast<float4*>(Ahi + off) = h4;
                *reinterpret_cast<float4*>(Alo + off) = l4;
              }
            }
          }
        }
      }
      // B operand: thread -> costate component ct of the tile, all 16 rows
      {
        const uint32_t rs = it % WG_RING;
        if (good) good = qptc::mbar_wait(&raw_full[rs], (it / WG_RING) & 1);
        float lv[WKC];
        const float* rr = raw + rs * (WKC * 256);
#pragma unroll
        for (int t = 0; t < WKC; ++t) lv[t] = (good && t < nvalid) ? rr[t * 256 + ct] : 0.f;
        __syncwarp();
        if (lane == 0) qptc::mbar_arrive(&raw_free[rs]);
        if (H16) {
#pragma unroll
          for (int g8 = 0; g8 < WKC / 8; ++g8) {
            uint4 h8, l8;
            pack_h8(lv + 8 * g8, sL, h8, l8);
            const uint32_t off = core_off_w16(ct, g8 * 8);
            *reinterpret_cast<uint4*>(sB + off) = h8;
            *reinterpret_cast<uint4*>(sB + 256 * WKC * 2 + off) = l8;
          }
        } else {
          float* Bhi = reinterpret_cast<float*>(sB);
          float* Blo = Bhi + 256 * WKC;
#pragma unroll
          for (int g4 = 0; g4 < WKC / 4; ++g4) {
            float4 h4, l4;
            qptc::split_tf32_fast(lv[4 * g4], h4.x, l4.x);
            qptc::split_tf32_fast(lv[4 * g4 + 1], h4.y, l4.y);
            qptc::split_tf32_fast(lv[4 * g4 + 2], h4.z, l4.z);
            qptc::split_tf32_fast(lv[4 * g4 + 3], h4.w, l4.w);
            const uint32_t off = core_off16(ct, g4 * 4) / 4;
            *reinterpret_cast<float4*>(Bhi + off) = h4;
            *reinterpret_cast<float4*>(Blo + off) = l4;
          }
        }
      }
      qptc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) qptc::mbar_arrive(&stage_full[crew]);
      if ((vs + 1 + choff) % a.fl == 0 || vs + 1 == slen) {
        // the chunk's last step: drain once its MMAs (and so all earlier ones) finished
        if (good) good = qptc::mbar_wait(&mma_done[crew], cnt & 1);
        if (good) {
          qptc::fence_after();
          flush((vs + choff) / a.fl > 0, false, slot, tile);
        }
        // a segment's first drain stores, later ones add (in any order): the next chunk's drain
        // (another crew) must see the stores
        if ((vs + choff) / a.fl == 0) __threadfence();
        qptc::fence_before();
        __syncwarp();
        if (lane == 0) qptc::mbar_arrive(acc_free);
      }
      ok = __all_sync(0xffffffffu, good);
    }
    // a crew that stopped early tells its other warps through the barrier it left them in:
    // they time out on their own waits; the status records the failure
    if (!ok && lane == 0) atomicExch(a.status, 6);
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, tcols);
}

}  // namespace qpd
