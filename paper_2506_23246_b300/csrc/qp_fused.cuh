// qp_fused.cuh -- forward contraction of the fused-unitary path with the pointwise stage
// (readout, head, loss terms, cotangents, costates) as its tensor-memory epilogue, n = 7, 8.
#pragma once
#include <cuda.h>   // CUtensorMap (the maps are encoded on the host)
#include "qp_dense.cuh"

namespace qpd {

// ------------------------------------------------------------------------- fused forward + costates
// For n <= 8 a 128-row tile's whole output row (2^(n+1) <= 512 FP32 columns) stays in tensor
// memory, so the pointwise stage runs as the epilogue of the forward contraction and the
// states never reach HBM: readout z_i = <phi|Z_i|phi>, d z_i/dv_d = 2 Re<phi_d|Z_i|phi> (the
// readout of the forward-mode tangents), the linear head, the loss terms and cotangents of
// the point, and the costates
//   lambda_0 = O phi_0 + sum_d O_d phi_d,  lambda_d = O_d phi_0,  O = sum_i zbar_i Z_i
// (Z_i diagonal: O is a per-amplitude sign sum), written in place of the states.
// Tile rows: collocation tiles hold 32 points x 4 vectors (row = 4 point + vector, the order of
// the costate rows in HBM), so a point's four rows sit in one lane quad of a warp and every
// exchange between them is a shuffle; IC/BC tiles hold 128 points. Warps w and w + 4 read the
// same 32 rows, the two halves of the columns.
constexpr int F_STAGERS = 256;                 // operand generation + epilogue (8 warps)
constexpr int F_THREADS = F_STAGERS + 32;      // + one control warp (bulk copies, MMAs)
constexpr int F_MAXH = 5;       // embedding qubits above the 3 lowest index bits (n <= 8)


struct FusedArgs {
  const float* thetaJ;     // [P][n] float4 (theta, dtheta/dx, dtheta/dy, dtheta/dt)
  const __half* W16;       // [dim / HKC][nc][2 (hi, lo)][256 x HKC] FP16 operand pairs of W * W16_SCALE
  float* lam;              // costates (output), blocked layout [2^(n+1) / 256][rtot][256]
  int64_t rtot;
  const float* head;       // W[3][m], b[3]
  int32_t n, m;
  const float* pts[3];
  int64_t npts[3], pt_base[3];
  int64_t tile_end[3];     // cumulative tiles: collocation tiles of 32 points, IC/BC of 128
  QPProblemDev pb;
  const int32_t* counts;
  double* blk_loss;
  float* blk_grad;
  int32_t loss_stride, grad_stride, nE, nblk;
  int32_t* status;
  int32_t* scal;           // [2] float bits (atomic max): row bound of the product states, max |lambda|
  int32_t use_tma;         // 1: costates leave through tensor-map bulk stores (maps valid), 0: plain stores
  uint32_t wait_limit;     // polls of the pipeline waits (0: QP_MBAR_LIMIT); the drain waits that
                           // let in-flight copies and MMAs finish always keep QP_MBAR_LIMIT
  // symmetry penalty (Eq. 18): field cotangents added to the collocation points' (gsym,
  // [npts[0]][3]) and given outright for the rows of set 2 from nbc on, the mirrored points
  // (gext, [npts[2] - nbc][3]); both null without the penalty
  const float* gsym;
  const float* gext;
  int64_t nbc;
};

// Tensor-map bulk store of one staged 128-row x 32-column chunk (bulk group of this thread).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* m, const void* src, int x, int y, int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(m), "r"(x),
               "r"(y), "r"(z), "r"(qptc::smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// The bulk stores issued by this thread have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// All but the most recent bulk group of this thread have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_but1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

// Shared memory: two A stages (FP16 hi, lo), a three-slot ring of W blocks (copies run two
// K-steps ahead, across tile boundaries), and the persistent head/loss/barrier block. The
// epilogue's readout buffers and the second costate staging buffer live in the W slot of the
// tile's last K-step (idle until that slot's next copy, issued after the epilogue) when it is
// large enough, else in a region of their own; the first staging buffer is the A stages.
struct FusedSmem {
  int a_bytes, w_bytes, wbase, epi, zp, zb, st2, hw, sloss, hsum, rsc, bars, total;
  bool epi_in_w;
};
constexpr int F_STG_BYTES = 2 * TM * 32 * 4;   // one 128-row x 32-column chunk per column half
constexpr int F_EPI_BYTES = 16384 + F_STG_BYTES;
__host__ __device__ inline FusedSmem fused_smem(int n, int nt) {
  FusedSmem f;
  const int nc = (2 << n) / 256;
  f.a_bytes = TM * HKC * 2;
  f.w_bytes = nc * 2 * 256 * HKC * 2;
  f.wbase = 2 * 2 * f.a_bytes;
  int o = f.wbase + 3 * f.w_bytes;
  f.hw = o; o += (3 * QP_MAXQ + 3) * 4 + 4;       // head weights
  o = (o + 15) / 16 * 16;
  f.sloss = o; o += (QP_NLP + nt) * 8;
  o = (o + 15) / 16 * 16;
  f.hsum = o; o += (3 * QP_MAXQ + 3) * 4 + 4;
  o = (o + 15) / 16 * 16;
  f.rsc = o; o += TM * 4;                         // per-row unscale factors of the tile
  f.bars = o; o += 128;                           // w_full[3], mma_done[2], tensor-memory slot
  f.epi_in_w = f.w_bytes >= F_EPI_BYTES;
  if (!f.epi_in_w) { o = (o + 1023) / 1024 * 1024; f.epi = o; o += F_EPI_BYTES; }
  else f.epi = -1;
  // offsets inside the epilogue block (1024-byte aligned, as the swizzled staging needs)
  f.zp = 0;                                       // readout partials [half][row][i]
  f.zb = f.zp + 2 * TM * QP_MAXQ * 4;             // sign-sum coefficients [row][i]
  f.st2 = 16384;                                  // second costate staging buffer
  f.total = o;
  return f;
}

// bar.sync is the aligned form: the warp is reconverged before it.
__device__ __forceinline__ void named_bar(int id) {
  __syncwarp();
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(128) : "memory");
}
// Barrier over the staging warps only (the control warp never joins it).
__device__ __forceinline__ void stagers_bar() {
  __syncwarp();
  asm volatile("bar.sync %0, %1;" ::"r"(3), "r"(F_STAGERS) : "memory");
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// tm_c, tm_i, tm_b: the costate rows of the collocation, IC and BC sets as (column, row,
// 256-column block); tiles that run past a set's rows are clipped by the maps.
// NQ = n (7 or 8, equal to a.n): the qubit count fixes the bit positions of the embedding
// tables, the readout sign sums and the costate sign sums at compile time.
template <int NQ>
__global__ void __launch_bounds__(F_THREADS, 1) dense_fused_fwd_kernel(FusedArgs a, const __grid_constant__ CUtensorMap tm_c,
                                                                       const __grid_constant__ CUtensorMap tm_i,
                                                                       const __grid_constant__ CUtensorMap tm_b) {
  static_assert(NQ == 7 || NQ == 8, "the fused kernel holds a tile's 2^(n+1) columns in tensor memory");
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int n = NQ, dim = 1 << n;
  const int m = a.m, nt = a.pb.energy_nt;
  constexpr int nc = (2 << n) / 256;
  const FusedSmem L = fused_smem(n, nt);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ws = warp & 3, hh = warp >> 2;        // tensor-memory lane group, column half
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* w_full = bars;          // [3] W ring slot landed
  uint64_t* mma_done = bars + 3;    // [2] tensor-core work of an A stage finished (commit)
  uint64_t* a_full = bars + 5;      // [2] A operand of a stage written (8 staging warps)
  uint64_t* acc_free = bars + 7;    // tile epilogue done with tensor memory (8 staging warps)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.bars + 64);
  const bool ctrl = warp == F_STAGERS / 32;
  float* hw = reinterpret_cast<float*>(sm + L.hw);
  double* sloss = reinterpret_cast<double*>(sm + L.sloss);
  float* hsum = reinterpret_cast<float*>(sm + L.hsum);
  const uint32_t tcols = 2u << n;
  if (warp == 0) qptc::tmem_alloc(tslot, tcols);
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) qptc::mbar_init(&bars[i], 1);
    for (int i = 5; i < 8; ++i) qptc::mbar_init(&bars[i], F_STAGERS / 32);
  }
  for (int i = tid; i < 3 * m + 3; i += blockDim.x) { hw[i] = a.head[i]; hsum[i] = 0.f; }
  for (int i = tid; i < QP_NLP + nt; i += blockDim.x) sloss[i] = 0.0;
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = qptc::idesc(0, TM, 256);   // FP16 x FP16 -> FP32
  const int nkc = dim / HKC;
  float* rsc = reinterpret_cast<float*>(sm + L.rsc);
  const int arow = tid & (TM - 1), khalf = tid >> 7;
  const int r = ws * 32 + lane;                   // tile row read from tensor memory
  const int half_cols = dim;                      // 2 dim columns split between two halves
  // per-thread running sums over all tiles (point threads only), compensated FP32
  CSum lacc[QP_NLP];
  float hg[3][QP_MAXQ], hb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    hb[c] = 0.f;
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) hg[c][i] = 0.f;
  }
  bool ok = true;
  uint32_t it = 0;
  int64_t last_copy = -1, last_commit = -1;
  const uint32_t lim = a.wait_limit ? a.wait_limit : QP_MBAR_LIMIT;
  const int64_t T2 = a.tile_end[2];
  const int64_t ntl = (int64_t)blockIdx.x < T2 ? (T2 - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t total = ntl * nkc;
  if (ctrl) {
    // ---- control thread: W two K-steps ahead, MMAs as soon as a stage's A is written
    if (lane == 0) {
      const uint32_t wblk = 256 * HKC * 2;
      for (int j = 0; j < 2 && j < total; ++j) {
        qptc::mbar_arrive_expect_tx(&w_full[j], L.w_bytes);
        qptc::bulk_g2s(sm + L.wbase + j * L.w_bytes, a.W16 + (int64_t)(j % nkc) * (L.w_bytes / 2), L.w_bytes,
                       &w_full[j]);
        last_copy = j;
      }
      for (int64_t t = 0; t < ntl && ok; ++t) {
        for (int kc = 0; kc < nkc && ok; ++kc, ++it) {
          const uint32_t st = it & 1, wsl = it % 3;
          // the previous tile's epilogue must be done with tensor memory (and with W slot it - 1)
          if (kc == 0 && t > 0) ok = qptc::mbar_wait(acc_free, (uint32_t)(t - 1) & 1, lim);
          if (ok) ok = qptc::mbar_wait(&w_full[wsl], (it / 3) & 1, lim);
          if (ok) ok = qptc::mbar_wait(&a_full[st], (it >> 1) & 1, lim);
          if (!ok) break;
          qptc::fence_after();
          const uint32_t sa = qptc::smem_u32(sm + st * 2 * L.a_bytes), sw = qptc::smem_u32(sm + L.wbase + wsl * L.w_bytes);
#pragma unroll
          for (int ks = 0; ks < HKC / 16; ++ks) {
            const uint64_t ah = qptc::desc_kmajor(sa + ks * 256, 128, (HKC / 8) * 128);
            const uint64_t al = qptc::desc_kmajor(sa + L.a_bytes + ks * 256, 128, (HKC / 8) * 128);
            for (int c = 0; c < nc; ++c) {
              const uint64_t wh = qptc::desc_kmajor(sw + c * 2 * wblk + ks * 256, 128, (HKC / 8) * 128);
              const uint64_t wl = qptc::desc_kmajor(sw + c * 2 * wblk + wblk + ks * 256, 128, (HKC / 8) * 128);
              const uint32_t dt = tmem + c * 256;
              qptc::mma_f16(dt, ah, wh, id, (kc > 0 || ks > 0) ? 1u : 0u);
              qptc::mma_f16(dt, ah, wl, id, 1u);
              qptc::mma_f16(dt, al, wh, id, 1u);
            }
          }
          qptc::commit(&mma_done[st]);
          last_commit = it;
          if ((int64_t)it + 2 < total) {
            const uint32_t j = it + 2, js = j % 3;
            if (it >= 1) ok = qptc::mbar_wait(&mma_done[(it - 1) & 1], ((it - 1) >> 1) & 1, lim);
            if (!ok) break;
            // W slot js last held step it - 1 and, at a tile end, that tile's epilogue buffers:
            // copies into it are issued only after acc_free (above) for the first step of a tile
            qptc::fence_proxy_async();
            qptc::mbar_arrive_expect_tx(&w_full[js], L.w_bytes);
            qptc::bulk_g2s(sm + L.wbase + js * L.w_bytes, a.W16 + (int64_t)((kc + 2) % nkc) * (L.w_bytes / 2),
                           L.w_bytes, &w_full[js]);
            last_copy = j;
          }
        }
      }
      if (!ok) {
        atomicExch(a.status, 6);
        for (int64_t j = last_copy - 2 < 0 ? 0 : last_copy - 2; j <= last_copy; ++j)
          qptc::mbar_wait(&w_full[j % 3], (uint32_t)(j / 3) & 1);
        if (last_commit >= 0) qptc::mbar_wait(&mma_done[last_commit & 1], ((uint32_t)last_commit >> 1) & 1);
      }
    }
  } else
  for (int64_t tile = blockIdx.x; tile < T2 && ok; tile += gridDim.x) {
    int set;
    int64_t p0;
    if (tile < a.tile_end[0]) { set = 0; p0 = tile * 32; }
    else if (tile < a.tile_end[1]) { set = 1; p0 = (tile - a.tile_end[0]) * TM; }
    else { set = 2; p0 = (tile - a.tile_end[1]) * TM; }
    const bool nv4 = set == 0;
    const int64_t np = a.npts[set], base = a.pt_base[set];
    // ---- embedding tables of the A row generated by this thread
    const int s_a = nv4 ? (arow & 3) : 0;                 // row = 4 point + vector
    const int64_t pa = p0 + (nv4 ? (arow >> 2) : arow);
    const int64_t pac = pa < np ? pa : np - 1;
    const float4* tj = reinterpret_cast<const float4*>(a.thetaJ) + (base + pac) * n;
    float Lo[8], Lod[8];
    float jsum = 0.f;   // sum over qubits of |J| along this row's direction
#pragma unroll
    for (int t = 0; t < 8; ++t) { Lo[t] = 1.f; Lod[t] = 0.f; }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4 tq = __ldg(tj + (n - 1 - b));
      float sn, cs;
      sincosf(0.5f * tq.x, &sn, &cs);
      const float J = s_a == 0 ? 0.f : (s_a == 1 ? tq.y : (s_a == 2 ? tq.z : tq.w));
      jsum += fabsf(J);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const bool bit = (t >> b) & 1;
        const float f = bit ? sn : cs, d = bit ? 0.5f * cs : -0.5f * sn;
        Lod[t] = Lod[t] * f + Lo[t] * d * J;
        Lo[t] *= f;
      }
    }
    float hc[F_MAXH], hs[F_MAXH], hj[F_MAXH];
#pragma unroll
    for (int q = 0; q < F_MAXH; ++q) {
      hc[q] = 1.f; hs[q] = 0.f; hj[q] = 0.f;
      if (q < n - 3) {
        const float4 tq = __ldg(tj + q);
        sincosf(0.5f * tq.x, &hs[q], &hc[q]);
        hj[q] = s_a == 0 ? 0.f : (s_a == 1 ? tq.y : (s_a == 2 ? tq.z : tq.w));
        jsum += fabsf(hj[q]);
      }
    }
    // FP16 operand scale of this row (a power of two): |R_0| <= 1 and |R_d| <= sum_q |J_q| / 2
    // (each product-rule term carries one derivative factor of size at most |J| / 2), so the
    // scaled row stays below 2^13; the epilogue takes the scales back out of the accumulators.
    float rs;
    {
      const float bnd = s_a == 0 ? 1.f : 0.5f * jsum;
      int eb = 0;
      if (bnd > 0.f) frexpf(bnd, &eb);
      const int e = bnd > 0.f ? max(-100, min(100, 13 - eb)) : 0;
      rs = ldexpf(1.f, e);
      if (khalf == 0) rsc[arow] = ldexpf(1.f, -e) * (1.f / W16_SCALE);
      // the weight-gradient contraction scales all product-state rows by one bound
      const float wb = warp_max_f(bnd);
      if (lane == 0) atomicMax(a.scal, __float_as_int(wb));
    }
    // ---- forward contraction: TMEM[row][2j + re/im] = sum_k R[row][k] W[2j + re/im][k]
    for (int kc = 0; kc < nkc; ++kc, ++it) {
      const uint32_t st = it & 1;
      unsigned char* sA = sm + st * 2 * L.a_bytes;
      if (it >= 2 && ok) ok = qptc::mbar_wait(&mma_done[st], ((it - 2) >> 1) & 1, lim);
      if (ok) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          // basis indices k = kc * 32 + khalf * 16 + g * 8 + t: bits 0-2 from the tables, the
          // rest from H
          const int hbits = kc * 4 + khalf * 2 + g;
          float H = 1.f, Hd = 0.f;
#pragma unroll
          for (int q = 0; q < F_MAXH; ++q) {
            if (q < n - 3) {
              const bool bit = (hbits >> (n - 4 - q)) & 1;
              const float f = bit ? hs[q] : hc[q], d = bit ? 0.5f * hc[q] : -0.5f * hs[q];
              Hd = Hd * f + H * d * hj[q];
              H *= f;
            }
          }
          // FP16 pair of the scaled value: x = hi + lo (lo = the rounding remainder of hi)
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float x[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int t = 2 * e + u;
              x[u] = rs * (s_a == 0 ? H * Lo[t] : Hd * Lo[t] + H * Lod[t]);
            }
            const __half2 h2 = __floats2half2_rn(x[0], x[1]);
            const float2 hf = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(x[0] - hf.x, x[1] - hf.y);
            hw[e] = *reinterpret_cast<const uint32_t*>(&h2);
            lw[e] = *reinterpret_cast<const uint32_t*>(&l2);
          }
          const uint32_t off = core_off_h(arow, khalf * 16 + g * 8);
          *reinterpret_cast<uint4*>(sA + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(sA + L.a_bytes + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      }
      qptc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) qptc::mbar_arrive(&a_full[st]);
    }
    ok = qptc::bar_and(3, F_STAGERS, ok && qptc::mbar_wait(&mma_done[(it - 1) & 1], ((it - 1) >> 1) & 1, lim));
    if (!ok) break;
    qptc::fence_after();
    const float us = rsc[r];   // this thread's tensor-memory row: back to unscaled amplitudes
    // epilogue buffers: the W slot of the tile's last step (or their own region)
    unsigned char* epi = L.epi_in_w ? sm + L.wbase + ((it - 1) % 3) * L.w_bytes : sm + L.epi;
    float* zp = reinterpret_cast<float*>(epi + L.zp);
    const int s_r = nv4 ? (lane & 3) : 0;     // vector of this thread's row r = 4 point + vector
    const int q0 = lane & ~3;                 // the lane of the row's point with vector 0
    float* zbs = reinterpret_cast<float*>(epi + L.zb);
    // ---- pass 1: readout partial sums over this thread's half of the columns
    float acc[QP_MAXQ];
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) acc[i] = 0.f;
    for (int cc = 0; cc < half_cols; cc += 32) {
      const int col = hh * half_cols + cc;
      float v[32];   // scaled amplitudes: the row scale comes out of the partial sums below
      qptc::tmem_ld32(tmem + ((uint32_t)(ws * 32) << 16) + col, v);
      float y[16];
      if (nv4) {
        // the point's four rows sit in one lane quad: phi_0 comes from the quad's first lane
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float xa = __shfl_sync(0xffffffffu, v[2 * e], q0), xb = __shfl_sync(0xffffffffu, v[2 * e + 1], q0);
          y[e] = s_r == 0 ? v[2 * e] * v[2 * e] + v[2 * e + 1] * v[2 * e + 1] : 2.f * (v[2 * e] * xa + v[2 * e + 1] * xb);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) y[e] = v[2 * e] * v[2 * e] + v[2 * e + 1] * v[2 * e + 1];
      }
      // total and the four single-bit sign sums over the 16 amplitudes of the chunk, by
      // pairwise sums and differences (bit b: S_b = sum over bit b clear - sum over bit b set)
      float S[4];
      float s8[8], s4[4];
      {
        float d = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) { s8[k] = y[2 * k] + y[2 * k + 1]; d += y[2 * k] - y[2 * k + 1]; }
        S[0] = d;
        d = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) { s4[k] = s8[2 * k] + s8[2 * k + 1]; d += s8[2 * k] - s8[2 * k + 1]; }
        S[1] = d;
        S[2] = (s4[0] - s4[1]) + (s4[2] - s4[3]);
        S[3] = (s4[0] + s4[1]) - (s4[2] + s4[3]);
      }
      const float T = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      const int j0 = col >> 1;
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i) {
        if (i < m) {
          const int pbit = n - 1 - i;
          const float sv = pbit == 0 ? S[0] : pbit == 1 ? S[1] : pbit == 2 ? S[2] : pbit == 3 ? S[3]
                         : (((j0 >> pbit) & 1) ? -T : T);
          acc[i] += sv;
        }
      }
    }
    {
      // y is a product of this row's amplitudes with its own (vector 0) or its point's vector-0
      // row's amplitudes: one factor of each row scale
      const float us0 = __shfl_sync(0xffffffffu, us, q0);
      const float yf = us * (nv4 && s_r != 0 ? us0 : us);
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i)
        if (i < m) zp[(hh * TM + r) * QP_MAXQ + i] = acc[i] * yf;
    }
    stagers_bar();
    // ---- point stage: head, loss terms, cotangents, sign-sum coefficients. Collocation
    // tiles: the four lanes of a point (rows 4 point + vector) share the point's loss terms and
    // each forms the cotangent of its own row; IC/BC tiles: one point per lane.
    if (warp < 4) {
      const int pl = nv4 ? (r >> 2) : r;
      const int row0 = nv4 ? pl * 4 : pl;
      const int64_t pp = p0 + pl;
      const bool active = pp < np;
      const int64_t ppc = active ? pp : np - 1;
      float z[QP_MAXQ], dz[3][QP_MAXQ];
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i) {
        z[i] = 0.f; dz[0][i] = dz[1][i] = dz[2][i] = 0.f;
        if (i < m) {
          z[i] = zp[row0 * QP_MAXQ + i] + zp[(TM + row0) * QP_MAXQ + i];
          if (nv4) {
#pragma unroll
            for (int d = 0; d < 3; ++d)
              dz[d][i] = zp[(row0 + d + 1) * QP_MAXQ + i] + zp[(TM + row0 + d + 1) * QP_MAXQ + i];
          }
        }
      }
      float f[3], D[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float accf = hw[3 * m + c], ad[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < QP_MAXQ; ++i)
          if (i < m) {
            const float w = hw[c * m + i];
            accf += w * z[i];
#pragma unroll
            for (int d = 0; d < 3; ++d) ad[d] += w * dz[d][i];
          }
        f[c] = accf;
#pragma unroll
        for (int d = 0; d < 3; ++d) D[c][d] = ad[d];
      }
      const float* xp = a.pts[set] + ppc * 3;
      float g[3], gD[3][3];
      float lt[QP_NLP], ev;
      int slice;
      // rows of set 2 past the boundary points are mirrored points with given cotangents
      const bool given = set == 2 && a.gext != nullptr && pp >= a.nbc;
      const int64_t npl = set == 2 && a.gext != nullptr ? a.nbc : np;
      qpk::point_loss_terms(a.pb, set, ppc, npl, a.counts, __ldg(xp), __ldg(xp + 1), f, D, active && !given, lt, slice,
                            ev, g, gD);
      if (given && active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) g[c] = __ldg(a.gext + (pp - a.nbc) * 3 + c);
      }
      if (set == 0 && a.gsym != nullptr && active) {
#pragma unroll
        for (int c = 0; c < 3; ++c) g[c] += __ldg(a.gsym + pp * 3 + c);
      }
      if (s_r != 0) ev = 0.f;   // each point once
      if (s_r == 0) {
#pragma unroll
        for (int i = 0; i < QP_NLP; ++i) lacc[i].add(lt[i]);
#pragma unroll
        for (int c = 0; c < 3; ++c) hb[c] += g[c];
      }
      // energy slices: one FP64 shared add per warp when the warp's points share a slice
      const int s0 = __shfl_sync(0xffffffffu, slice, 0);
      if (__all_sync(0xffffffffu, slice == s0)) {
        const float evs = warp_sum_f(ev);
        if (lane == 0 && s0 >= 0) atomicAdd(&sloss[QP_NLP + s0], (double)evs);
      } else if (slice >= 0 && s_r == 0) {
        atomicAdd(&sloss[QP_NLP + slice], (double)ev);
      }
      // this row's cotangent weights: zbar (vector 0) or zbar_d (vector d), and its share of the
      // head gradient
      float gs[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) gs[c] = s_r == 0 ? g[c] : (s_r == 1 ? gD[c][0] : (s_r == 2 ? gD[c][1] : gD[c][2]));
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i) {
        if (i < m) {
          const float zs = s_r == 0 ? z[i] : (s_r == 1 ? dz[0][i] : (s_r == 2 ? dz[1][i] : dz[2][i]));
          float zb = 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float w = hw[c * m + i];
            zb += w * gs[c];
            hg[c][i] += gs[c] * zs;
          }
          zbs[r * QP_MAXQ + i] = zb;
        }
      }
    }
    stagers_bar();
    // ---- pass 2: costates of this thread's row, written over the state rows
    {
      float coef[QP_MAXQ], cb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i) {
        coef[i] = i < m ? zbs[r * QP_MAXQ + i] : 0.f;
        const int pbit = n - 1 - i;
        if (i < m && pbit < 4) {
          if (pbit == 0) cb[0] = coef[i];
          else if (pbit == 1) cb[1] = coef[i];
          else if (pbit == 2) cb[2] = coef[i];
          else cb[3] = coef[i];
        }
      }
      const float t01[4] = {cb[0] + cb[1], -cb[0] + cb[1], cb[0] - cb[1], -cb[0] - cb[1]};
      const float t23[4] = {cb[2] + cb[3], -cb[2] + cb[3], cb[2] - cb[3], -cb[2] - cb[3]};
      const int64_t grow0 = lam_row(set, p0, 0, a.npts[0], base);   // first costate row of the tile
      float lmax = 0.f;   // largest costate magnitude of this thread (FP16 scale of the next contractions)
      for (int cc = 0; cc < half_cols; cc += 32) {
        const int col = hh * half_cols + cc;
        const int j0 = col >> 1;
        float Bs = 0.f;
#pragma unroll
        for (int i = 0; i < QP_MAXQ; ++i) {
          const int pbit = n - 1 - i;
          if (i < m && pbit >= 4) Bs += ((j0 >> pbit) & 1) ? -coef[i] : coef[i];
        }
        float O[16], u01[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) u01[e] = Bs + t01[e];
#pragma unroll
        for (int e = 0; e < 16; ++e) O[e] = u01[e & 3] + t23[e >> 2];
        float v[32];   // scaled amplitudes: the row scales are folded into O below
        qptc::tmem_ld32(tmem + ((uint32_t)(ws * 32) << 16) + col, v);
        // [128 rows][8] float4 staging, two buffers in turn: the A stages (idle during the
        // epilogue) and a buffer beside the readout partials
        float4* stg = reinterpret_cast<float4*>(((cc >> 5) & 1) ? epi + L.st2 : sm) + hh * 1024;
        const bool issuer = ws == 0 && lane == 0;
        // the store of the chunk before last (same buffer) has read the staging; 16-byte piece
        // e of row r is staged at e ^ (r mod 8)
        if (a.use_tma && issuer) bulk_wait_read_but1();
        named_bar(1 + hh);
        if (nv4) {
          // lambda_s = O_s phi_0 for s >= 1 (phi_0 from the quad's first lane), then
          // lambda_0 = sum_s O_s phi_s over the quad, reduced so that lane s keeps columns
          // 8s .. 8s + 7 of it
          const float us0 = __shfl_sync(0xffffffffu, us, q0);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            float x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = __shfl_sync(0xffffffffu, v[4 * e + u], q0);
            const float oa = O[2 * e] * us0, ob = O[2 * e + 1] * us0;
            const float4 o4 = make_float4(oa * x[0], oa * x[1], ob * x[2], ob * x[3]);
            if (s_r != 0) {
              stg[r * 8 + (e ^ (r & 7))] = o4;
              lmax = fmaxf(lmax, fmaxf(fmaxf(fabsf(o4.x), fabsf(o4.y)), fmaxf(fabsf(o4.z), fabsf(o4.w))));
            }
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) O[e] *= us;
#pragma unroll
          for (int k = 0; k < 32; ++k) v[k] *= O[k >> 1];
          const bool up = (s_r & 2) != 0, lo = (s_r & 1) != 0;
          float kept[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float keep = up ? v[16 + k] : v[k], send = up ? v[k] : v[16 + k];
            kept[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
          }
          float l0[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float keep = lo ? kept[8 + k] : kept[k], send = lo ? kept[k] : kept[8 + k];
            l0[k] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
          }
          const int rq = r & ~3;
#pragma unroll
          for (int j2 = 0; j2 < 2; ++j2) {
            const float4 o4 = make_float4(l0[4 * j2], l0[4 * j2 + 1], l0[4 * j2 + 2], l0[4 * j2 + 3]);
            stg[rq * 8 + ((2 * s_r + j2) ^ (rq & 7))] = o4;
            lmax = fmaxf(lmax, fmaxf(fmaxf(fabsf(o4.x), fabsf(o4.y)), fmaxf(fabsf(o4.z), fabsf(o4.w))));
          }
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) O[e] *= us;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float4 o4 = make_float4(O[2 * e] * v[4 * e], O[2 * e] * v[4 * e + 1], O[2 * e + 1] * v[4 * e + 2],
                                          O[2 * e + 1] * v[4 * e + 3]);
            stg[r * 8 + (e ^ (r & 7))] = o4;
            lmax = fmaxf(lmax, fmaxf(fmaxf(fabsf(o4.x), fabsf(o4.y)), fmaxf(fabsf(o4.z), fabsf(o4.w))));
          }
        }
        if (a.use_tma) {
          // one thread of the half hands the chunk to a tensor-map bulk store
          qptc::fence_proxy_async();
          named_bar(1 + hh);
          if (issuer) {
            tma_store_3d(set == 0 ? &tm_c : (set == 1 ? &tm_i : &tm_b), stg, col & 255, (int)(nv4 ? p0 * 4 : p0), col >> 8);
            bulk_commit();
          }
        } else {
          // plain stores of 128-byte row segments, four rows per warp instruction
          named_bar(1 + hh);
          const int gt = ws * 32 + lane;
          const int nrows = (int)(nv4 ? (np - p0 < 32 ? (np - p0) * 4 : 128) : (np - p0 < TM ? np - p0 : TM));
          float* gbase = a.lam + (int64_t)(col >> 8) * a.rtot * 256 + grow0 * 256 + (col & 255);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int idx = i * 128 + gt, row = idx >> 3, c4 = idx & 7;
            if (row < nrows) *reinterpret_cast<float4*>(gbase + (int64_t)row * 256 + c4 * 4) = stg[row * 8 + (c4 ^ (row & 7))];
          }
        }
      }
      const float wl = warp_max_f(lmax);
      if (lane == 0) atomicMax(a.scal + 1, __float_as_int(wl));
      // the next tile's operands overwrite the staging: its last store must have read it
      if (a.use_tma && ws == 0 && lane == 0) bulk_wait_read();
    }
    // tensor memory and the W slot of this tile's last step are free again
    qptc::fence_before();
    stagers_bar();
    if (lane == 0) qptc::mbar_arrive(acc_free);
  }
  if (!ok && !ctrl && tid == 0) atomicExch(a.status, 6);
  // ---- block partials: loss sums (FP64) and head gradients
#pragma unroll
  for (int i = 0; i < QP_NLP; ++i) {
    const double v = warp_sum_d((double)lacc[i].s + (double)lacc[i].c);
    if (lane == 0 && warp < 4 && v != 0.0) atomicAdd(&sloss[i], v);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) {
      if (i < m) {
        const float v = warp_sum_f(hg[c][i]);
        if (lane == 0 && warp < 4) atomicAdd(&hsum[c * m + i], v);
      }
    }
    const float v = warp_sum_f(hb[c]);
    if (lane == 0 && warp < 4) atomicAdd(&hsum[3 * m + c], v);
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, tcols);
  for (int b = blockIdx.x; b < a.nblk; b += gridDim.x) {
    const bool mine = b == (int)blockIdx.x;
    double* bl = a.blk_loss + (int64_t)b * a.loss_stride;
    for (int i = tid; i < QP_NLP + nt; i += blockDim.x) bl[i] = mine ? sloss[i] : 0.0;
    float* bg = a.blk_grad + (int64_t)b * a.grad_stride;
    for (int i = tid; i < a.nE; i += blockDim.x) bg[i] = 0.f;
    for (int i = tid; i < 3 * m + 3; i += blockDim.x) bg[a.nE + i] = mine ? hsum[i] : 0.f;
  }
}

}  // namespace qpd
