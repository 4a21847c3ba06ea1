// qp_wgrad.cuh -- weight-gradient contraction G = sum over (point, vector) rows of
// R Lambda^H on the tensor cores (3xTF32), FP32 partials per row range.
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
// Persistent CTAs: CTA b owns tile b % tiles and a balanced range of steps; every `fl` steps
// (<= 512 rows, the FP32 accumulation length in tensor memory) the accumulator is added into
// the CTA's partial slot (a few FP32 adds per element, the slot stays in L2); the slots of
// all CTAs of a tile are summed later in compensated FP32.
//
// Pipeline of one step (3 block barriers): the costate rows arrive in a 4-slot shared-memory
// ring by bulk copies issued three steps ahead; the step's R tables were built during the
// previous step and their angle factors the step before. A step writes its A operand from the
// tables, builds the next tables and factors, reads its costate columns, starts the copy three
// steps ahead, splits the columns into the TF32 B operand, and one thread issues the MMAs.
constexpr int WKC = 16;

// Fire-and-forget vector add into global memory (performed at L2).
__device__ __forceinline__ void red_add_f4(float4* p, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
constexpr int WG_STAGERS = 512;                 // operand-staging threads (16 warps)
constexpr int WG_THREADS = WG_STAGERS + 32;       // + one control warp (copies, MMAs)
constexpr int WG_RING = 4;

struct WgArgs {
  const float* thetaJ;        // [P][n] float4 (theta, J_x, J_y, J_t)
  const float2* cs;           // [P][n] (cos, sin) of theta / 2
  const float* lam;           // costate rows: blocked [2 dim / 256][rtot][256] or rows [P][4][2 dim]
  int64_t rtot;               // rows of the blocked layout (0: row layout)
  float* part;                // [ngroups][dim][2 dim], one slot per CTA of a tile
  int32_t n;
  int64_t npts[3], pt_base[3];
  int64_t kc_end[3];          // cumulative 16-row step counts per set
  int32_t tiles, ngroups, spc, fl;  // tiles, CTAs per tile, flushes per CTA, steps per flush
  int32_t* status;
  const int32_t* scal;        // FP16 operands: [2] float bits, bound of |R|, max |lambda|
};

// Byte offset of 16-bit element (row r, K index k) in a K-major WKC-wide block (core matrices
// of 8 rows x 8 elements, K-adjacent ones 128 bytes apart, 8-row groups 256 bytes apart).
__host__ __device__ inline uint32_t core_off_w16(int r, int k) {
  return (uint32_t)((r >> 3) * (WKC / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}


struct WgSmem {
  int a_bytes, b_bytes, stage, raw, fac, tab, bars, total;
};
constexpr int WG_TAB4 = 16 * 32 + 16 * 8;                 // Lo [16 pts][32], H [16 pts][8] float4
constexpr int WG_FAC4 = 16 * QP_MAXQ * 2;                 // [16 pts][q][2] float4
__host__ __device__ inline int wg_mtc(int n) { return (1 << n) < 256 ? (1 << n) : 256; }
// esz: operand element size, 4 (TF32 pairs) or 2 (FP16 pairs)
__host__ __device__ inline WgSmem wg_smem(int n, int esz = 4) {
  WgSmem w;
  w.a_bytes = (wg_mtc(n) / TM) * 2 * TM * WKC * esz;   // hi, lo per M sub-tile
  w.b_bytes = 2 * 256 * WKC * esz;                     // hi, lo
  w.stage = w.a_bytes + w.b_bytes;
  int o = 2 * w.stage;
  w.raw = o; o += WG_RING * WKC * 256 * 4;           // costate columns of a step [16][256]
  w.fac = o; o += 2 * WG_FAC4 * 16;
  w.tab = o; o += 2 * WG_TAB4 * 16;
  // mma_done[2], raw_full[4], stage_full[2], raw_free[4], acc_free, tab_full[2], tab_free[2], tmem slot
  w.bars = o; o += 192;
  w.total = o;
  return w;
}
__host__ inline int wg_smem_bytes(int n, bool h16 = false) { return wg_smem(n, h16 ? 2 : 4).total; }

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

// Tables of one step: Lo over the five low qubits, H over the others for k = kbase + 32 j.
__device__ __forceinline__ void wg_tables(const float4* fac, float4* tab, int tid, int n, int ppc, int kbase,
                                          int nj) {
  float4* tlo = tab;
  float4* thi = tab + 16 * 32;
  for (int idx = tid; idx < ppc * 32; idx += WG_STAGERS / 2) {
    const int pl = idx >> 5, e = idx & 31;
    float4 p = make_float4(1.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int b = 4; b >= 0; --b) {
      const int q = n - 1 - b;
      p = wg_dmul(p, fac[(pl * n + q) * 2], fac[(pl * n + q) * 2 + 1], (e >> b) & 1);
    }
    tlo[idx] = p;
  }
  // the H entries start at the fifth warp of the group: the first four hold the Lo entries of
  // a collocation step, so no warp builds both
  for (int idx = (tid + WG_STAGERS / 4) & (WG_STAGERS / 2 - 1); idx < ppc * 8; idx += WG_STAGERS / 2) {
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

// H16: FP16 operand pairs (kind::f16, one K = 16 MMA per term) with one power-of-two scale
// per operand from the recorded ranges; else TF32 pairs (two K = 8 MMAs per term).
// NQ = n (7 .. 10, equal to a.n): the qubit count fixes the (point, qubit) slot arithmetic and
// the table loops at compile time.
template <bool H16, int NQ>
__global__ void __launch_bounds__(WG_THREADS, 1) dense_wgrad_gemm_kernel(WgArgs a) {
  static_assert(NQ >= 7 && NQ <= 10, "weight-gradient contraction: 7 to 10 qubits");
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int n = NQ, dim = 1 << n;
  const WgSmem L = wg_smem(n, H16 ? 2 : 4);
  float sR = 1.f, sL = 1.f;
  if (H16) {
    sR = pow2_scale(__int_as_float(__ldg(a.scal)));
    sL = pow2_scale(__int_as_float(__ldg(a.scal + 1)));
  }
  const float unsc = 1.f / (sR * sL);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool ctrl = warp == WG_STAGERS / 32;
  const int MTC = wg_mtc(n), msub = MTC / TM, nj = MTC / 32;
  const int tile = blockIdx.x % a.tiles, lb = blockIdx.x / a.tiles;
  const int nmt = dim / MTC;
  const int mtile = tile % nmt, ntile = tile / nmt;
  const int kbase = mtile * MTC;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* mma_done = bars;          // [2]  tensor-core work of a stage finished (commit)
  uint64_t* raw_full = bars + 2;      // [4]  costate rows of a ring slot landed
  uint64_t* stage_full = bars + 6;    // [2]  A and B operands of a stage written (16 warps)
  uint64_t* raw_free = bars + 8;      // [4]  ring slot read by the B-group (8 warps)
  uint64_t* acc_free = bars + 12;     // accumulator flushed (16 warps)
  uint64_t* tab_full = bars + 13;     // [2]  tables of a step written (A-group, 8 warps)
  uint64_t* tab_free = bars + 15;     // [2]  tables of a step read by the B-group (8 warps)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.bars + 136);
  float* raw = reinterpret_cast<float*>(sm + L.raw);
  float4* facb = reinterpret_cast<float4*>(sm + L.fac);
  float4* tabb = reinterpret_cast<float4*>(sm + L.tab);
  const uint32_t tcols = msub * 256;
  constexpr int NSW = WG_STAGERS / 32;
  if (warp == 0) qptc::tmem_alloc(tslot, tcols);
  if (tid == 0) {
    for (int i = 0; i < 6; ++i) qptc::mbar_init(&bars[i], 1);
    for (int i = 6; i < 8; ++i) qptc::mbar_init(&bars[i], NSW);        // stage_full: all staging warps
    for (int i = 8; i < 12; ++i) qptc::mbar_init(&bars[i], NSW / 2);   // raw_free: B-group warps
    qptc::mbar_init(&bars[12], NSW);                                   // acc_free: all staging warps
    for (int i = 13; i < 17; ++i) qptc::mbar_init(&bars[i], NSW / 2);  // tab_full, tab_free
  }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const int64_t nkc = a.kc_end[2];
  const int64_t c0 = (int64_t)lb * nkc / a.ngroups, c1 = (int64_t)(lb + 1) * nkc / a.ngroups;
  const bool agrp = tid < WG_STAGERS / 2;   // A-group: R tables and A operand; B-group: costates
  const int kk = tid & (TM - 1), khalf = (tid >> 7) & 1;
  // (point, qubit) slot of this thread for the angle loads and factors: the group's last warp
  // first (a collocation step has 4 x n <= 32 of them), away from the warps building tables
  const int fid = (tid + 32) & (WG_STAGERS / 2 - 1);
  // two M sub-tiles: the B-group writes the second one's A operand from the same tables
  const bool bsplit = msub == 2;
  int64_t last_commit = -1, last_copy = -1;
  WgAng tjn{};  // A-group: angles of step c0 + it + 2
  if (c0 < c1) {
    if (!ctrl) {
      if (agrp) {
        int set, ppc, nv;
        int64_t p0;
        wg_step_geom(a, c0, set, p0, ppc, nv);
        wg_fac(facb, fid, n, ppc, wg_load_ang(a, c0, fid, n));
        if (c0 + 1 < c1) {
          int set1, ppc1, nv1;
          int64_t p01;
          wg_step_geom(a, c0 + 1, set1, p01, ppc1, nv1);
          wg_fac(facb + WG_FAC4, fid, n, ppc1, wg_load_ang(a, c0 + 1, fid, n));
        }
        if (c0 + 2 < c1) tjn = wg_load_ang(a, c0 + 2, fid, n);
      }
    } else if (lane == 0) {
      for (int j = 0; j < WG_RING - 1 && c0 + j < c1; ++j) {
        wg_copy_rows(a, c0 + j, ntile, raw + j * (WKC * 256), &raw_full[j]);
        last_copy = j;
      }
    }
  }
  __syncthreads();
  if (c0 < c1 && !ctrl && agrp) {
    int set, ppc, nv;
    int64_t p0;
    wg_step_geom(a, c0, set, p0, ppc, nv);
    wg_tables(facb, tabb, tid, n, ppc, kbase, nj);
  }
  __syncthreads();
  bool ok = true;
  if (ctrl) {
    // ---- control thread: bulk copies three steps ahead, MMAs when a stage is full
    if (lane == 0) {
      const uint32_t id = qptc::idesc(H16 ? 0 : 2, TM, 256);
      int slot = 0;
      bool fresh = true;
      uint32_t it = 0;
      for (int64_t kc = c0; kc < c1 && ok; ++kc, ++it) {
        const uint32_t st = it & 1;
        const int64_t j = it + WG_RING - 1;
        if (kc + WG_RING - 1 < c1) {
          if (j >= WG_RING) ok = qptc::mbar_wait(&raw_free[j % WG_RING], (uint32_t)((j - WG_RING) / WG_RING) & 1);
          if (!ok) break;
          qptc::fence_proxy_async();
          wg_copy_rows(a, kc + WG_RING - 1, ntile, raw + (j % WG_RING) * (WKC * 256), &raw_full[j % WG_RING]);
          last_copy = j;
        }
        if (fresh && slot > 0) ok = qptc::mbar_wait(acc_free, (uint32_t)(slot - 1) & 1);
        if (!ok) break;
        ok = qptc::mbar_wait(&stage_full[st], (it >> 1) & 1);
        if (!ok) break;
        qptc::fence_after();
        unsigned char* sA = sm + st * L.stage;
        const uint32_t sa = qptc::smem_u32(sA), sb = qptc::smem_u32(sA + L.a_bytes);
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
        qptc::commit(&mma_done[st]);
        last_commit = it;
        fresh = false;
        if ((kc - c0 + 1) % a.fl == 0 || kc + 1 == c1) {
          fresh = true;
          ++slot;
        }
      }
      if (!ok) {
        atomicExch(a.status, 6);
        // let every bulk copy and tensor-core operation of this CTA land before exiting
        for (int64_t j = last_copy - (WG_RING - 1) < 0 ? 0 : last_copy - (WG_RING - 1); j <= last_copy; ++j)
          qptc::mbar_wait(&raw_full[j % WG_RING], (uint32_t)(j / WG_RING) & 1);
        if (last_commit >= 0) qptc::mbar_wait(&mma_done[last_commit & 1], ((uint32_t)last_commit >> 1) & 1);
      }
    }
  } else {
    // ---- staging warps
    // epilogue of one partial: part[CTA slot] (+)= the MTC x 256 accumulator; every element
    // is read and written by the same thread at every flush
    auto flush = [&](bool add, bool zero) {
      const int g = warp & 3, qw = warp >> 2;          // lane group, quarter of the columns
      const int u = msub == 2 ? qw >> 1 : 0;            // M sub-tile read by this warp
      const int cbeg = msub == 2 ? (qw & 1) * 128 : qw * 64, ncols = msub == 2 ? 128 : 64;
      const int64_t krow = kbase + u * TM + g * 32 + lane;
      float* outp = a.part + (((int64_t)lb * dim) + krow) * (2 * dim) + ntile * 256 + cbeg;
      if (!zero) {
        float v[32];
        for (int c = 0; c < ncols; c += 32) {
          qptc::tmem_ld32(tmem + ((uint32_t)(g * 32) << 16) + u * 256 + cbeg + c, v);
          float4* o4 = reinterpret_cast<float4*>(outp + c);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float4 r = make_float4(unsc * v[4 * e], unsc * v[4 * e + 1], unsc * v[4 * e + 2], unsc * v[4 * e + 3]);
            if (add) red_add_f4(o4 + e, r);   // no return value: the flush does not wait on L2
            else o4[e] = r;
          }
        }
      } else {
        for (int c = 0; c < ncols; c += 4) *reinterpret_cast<float4*>(outp + c) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    int slot = 0;
    uint32_t it = 0;
    for (int64_t kc = c0; kc < c1 && ok; ++kc, ++it) {
      const uint32_t st = it & 1;
      unsigned char* sA = sm + st * L.stage;
      unsigned char* sB = sA + L.a_bytes;
      int set, ppc, nvalid;
      int64_t p0;
      wg_step_geom(a, kc, set, p0, ppc, nvalid);
      bool good = true;
      if (it >= 2) good = qptc::mbar_wait(&mma_done[st], ((it - 2) >> 1) & 1);
      if (agrp) {
        if (good) {
          // A operand of this step from its tables: thread -> (k, half of the rows), both M sub-tiles
          const float4* tlo = tabb + (it & 1) * WG_TAB4;
          const float4* thi = tlo + 16 * 32;
          const int e = kk & 31;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            if (u < (bsplit ? 1 : msub)) {
              const int j = (u * TM + kk) >> 5;
              float av[8];
              if (set == 0) {
#pragma unroll
                for (int pi = 0; pi < 2; ++pi) {
                  const int pl = khalf * 2 + pi;
                  const float4 h = thi[pl * 8 + j], l = tlo[pl * 32 + e];
                  av[4 * pi] = h.x * l.x;
                  av[4 * pi + 1] = h.y * l.x + h.x * l.y;
                  av[4 * pi + 2] = h.z * l.x + h.x * l.z;
                  av[4 * pi + 3] = h.w * l.x + h.x * l.w;
                }
              } else {
#pragma unroll
                for (int pi = 0; pi < 8; ++pi) {
                  const int pl = khalf * 8 + pi;
                  av[pi] = thi[pl * 8 + j].x * tlo[pl * 32 + e].x;
                }
              }
              if (H16) {
                uint4 h8, l8;
                pack_h8(av, sR, h8, l8);
                unsigned char* Ab = sA + u * 2 * (TM * WKC * 2);
                const uint32_t off = core_off_w16(kk, khalf * 8);
                *reinterpret_cast<uint4*>(Ab + off) = h8;
                *reinterpret_cast<uint4*>(Ab + TM * WKC * 2 + off) = l8;
              }
              float* Ahi = reinterpret_cast<float*>(sA + u * 2 * (TM * WKC * 4));
              float* Alo = Ahi + TM * WKC;
#pragma unroll
              for (int g4 = 0; g4 < (H16 ? 0 : 2); ++g4) {
                float4 h4, l4;
                qptc::split_tf32_fast(av[4 * g4], h4.x, l4.x);
                qptc::split_tf32_fast(av[4 * g4 + 1], h4.y, l4.y);
                qptc::split_tf32_fast(av[4 * g4 + 2], h4.z, l4.z);
                qptc::split_tf32_fast(av[4 * g4 + 3], h4.w, l4.w);
                const uint32_t off = core_off16(kk, khalf * 8 + g4 * 4) / 4;
                *reinterpret_cast<float4*>(Ahi + off) = h4;
                *reinterpret_cast<float4*>(Alo + off) = l4;
              }
            }
          }
          // tables of the next step (their buffer held the tables of step it - 1, which the
          // B-group may still be reading), factors of the step after
          if (kc + 1 < c1) {
            int set1, ppc1, nv1;
            int64_t p01;
            wg_step_geom(a, kc + 1, set1, p01, ppc1, nv1);
            if (bsplit && it >= 1) good = qptc::mbar_wait(&tab_free[(it + 1) & 1], ((it - 1) >> 1) & 1);
            if (good) wg_tables(facb + ((it + 1) & 1) * WG_FAC4, tabb + ((it + 1) & 1) * WG_TAB4, tid, n, ppc1, kbase, nj);
            if (bsplit) {
              __syncwarp();
              if (lane == 0) qptc::mbar_arrive(&tab_full[(it + 1) & 1]);
            }
          }
          if (kc + 2 < c1) {
            int set2, ppc2, nv2;
            int64_t p02;
            wg_step_geom(a, kc + 2, set2, p02, ppc2, nv2);
            wg_fac(facb + (it & 1) * WG_FAC4, fid, n, ppc2, tjn);
            if (kc + 3 < c1) tjn = wg_load_ang(a, kc + 3, fid, n);
          }
        }
      } else {
        if (bsplit) {
          // A operand of the second M sub-tile from this step's tables (written by the A-group
          // during the previous step; those of the first step before the loop)
          if (good && it >= 1) good = qptc::mbar_wait(&tab_full[it & 1], ((it - 1) >> 1) & 1);
          const int bo2 = tid - WG_STAGERS / 2;
          const int k2 = bo2 & (TM - 1), h2 = bo2 >> 7;
          const float4* tlo = tabb + (it & 1) * WG_TAB4;
          const float4* thi = tlo + 16 * 32;
          const int j = (TM + k2) >> 5, e = k2 & 31;
          float av[8];
          if (set == 0) {
#pragma unroll
            for (int pi = 0; pi < 2; ++pi) {
              const int pl = h2 * 2 + pi;
              const float4 h = thi[pl * 8 + j], l = tlo[pl * 32 + e];
              av[4 * pi] = h.x * l.x;
              av[4 * pi + 1] = h.y * l.x + h.x * l.y;
              av[4 * pi + 2] = h.z * l.x + h.x * l.z;
              av[4 * pi + 3] = h.w * l.x + h.x * l.w;
            }
          } else {
#pragma unroll
            for (int pi = 0; pi < 8; ++pi) {
              const int pl = h2 * 8 + pi;
              av[pi] = thi[pl * 8 + j].x * tlo[pl * 32 + e].x;
            }
          }
          __syncwarp();
          if (lane == 0) qptc::mbar_arrive(&tab_free[it & 1]);
          if (good) {
            if (H16) {
              uint4 h8, l8;
              pack_h8(av, sR, h8, l8);
              unsigned char* Ab = sA + 2 * (TM * WKC * 2);
              const uint32_t off = core_off_w16(k2, h2 * 8);
              *reinterpret_cast<uint4*>(Ab + off) = h8;
              *reinterpret_cast<uint4*>(Ab + TM * WKC * 2 + off) = l8;
            } else {
              float* Ahi = reinterpret_cast<float*>(sA + 2 * (TM * WKC * 4));
              float* Alo = Ahi + TM * WKC;
#pragma unroll
              for (int g4 = 0; g4 < 2; ++g4) {
                float4 h4, l4;
                qptc::split_tf32_fast(av[4 * g4], h4.x, l4.x);
                qptc::split_tf32_fast(av[4 * g4 + 1], h4.y, l4.y);
                qptc::split_tf32_fast(av[4 * g4 + 2], h4.z, l4.z);
                qptc::split_tf32_fast(av[4 * g4 + 3], h4.w, l4.w);
                const uint32_t off = core_off16(k2, h2 * 8 + g4 * 4) / 4;
                *reinterpret_cast<float4*>(Ahi + off) = h4;
                *reinterpret_cast<float4*>(Alo + off) = l4;
              }
            }
          }
        }
        // this step's costate columns (bulk-copied three steps ahead): component bo, 16 rows
        const uint32_t rs = it % WG_RING;
        if (good) good = qptc::mbar_wait(&raw_full[rs], (it / WG_RING) & 1);
        float lv[WKC];
        const int bo = tid - WG_STAGERS / 2;
        const float* rr = raw + rs * (WKC * 256);
#pragma unroll
        for (int t = 0; t < WKC; ++t) lv[t] = (good && t < nvalid) ? rr[t * 256 + bo] : 0.f;
        __syncwarp();
        if (lane == 0) qptc::mbar_arrive(&raw_free[rs]);
        if (H16) {
#pragma unroll
          for (int g8 = 0; g8 < WKC / 8; ++g8) {
            uint4 h8, l8;
            pack_h8(lv + 8 * g8, sL, h8, l8);
            const uint32_t off = core_off_w16(bo, g8 * 8);
            *reinterpret_cast<uint4*>(sB + off) = h8;
            *reinterpret_cast<uint4*>(sB + 256 * WKC * 2 + off) = l8;
          }
        }
        float* Bhi = reinterpret_cast<float*>(sB);
        float* Blo = Bhi + 256 * WKC;
#pragma unroll
        for (int g4 = 0; g4 < (H16 ? 0 : WKC / 4); ++g4) {
          float4 h4, l4;
          qptc::split_tf32_fast(lv[4 * g4], h4.x, l4.x);
          qptc::split_tf32_fast(lv[4 * g4 + 1], h4.y, l4.y);
          qptc::split_tf32_fast(lv[4 * g4 + 2], h4.z, l4.z);
          qptc::split_tf32_fast(lv[4 * g4 + 3], h4.w, l4.w);
          const uint32_t off = core_off16(bo, g4 * 4) / 4;
          *reinterpret_cast<float4*>(Bhi + off) = h4;
          *reinterpret_cast<float4*>(Blo + off) = l4;
        }
      }
      qptc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) qptc::mbar_arrive(&stage_full[st]);
      if ((kc - c0 + 1) % a.fl == 0 || kc + 1 == c1) {
        if (good) good = qptc::mbar_wait(&mma_done[st], (it >> 1) & 1);
        if (good) {
          qptc::fence_after();
          flush(slot > 0, false);
        }
        qptc::fence_before();
        __syncwarp();
        if (lane == 0) qptc::mbar_arrive(acc_free);
        ++slot;
      }
      // the A-group shares tables and factors across steps: one barrier per step over it
      if (agrp) ok = qptc::bar_and(1, WG_STAGERS / 2, good);
      else ok = __all_sync(0xffffffffu, good);
    }
    if (ok) {
      if (slot == 0) flush(false, true);   // no rows: the slot still joins the sum
    } else if (tid == 0) {
      atomicExch(a.status, 6);
    }
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, tcols);
}

}  // namespace qpd
