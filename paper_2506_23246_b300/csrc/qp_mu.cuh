// qp_mu.cuh -- back-projection mu = Re(U'^H lambda) on the tensor cores with the embedding
// gradients as its epilogue, n = 7, 8.
#pragma once
#include "qp_dense.cuh"

namespace qpd {

// ------------------------------------------------------------------------- mu + embedding gradients
// n <= 8: mu_s = Re(U'^H lambda_s) row by row on the tensor cores (A = costate rows, B = the
// transposed operand blocks), and the embedding gradients taken from tensor memory in the
// epilogue. With the flipped-factor identity d r / d theta_q [k] ~ sign_q(k) r[k ^ e_q]
// (the derivative of cos/sin(theta/2) is the other one, halved and signed), a row (p, s)
// contributes
//   C_q = sum_k sign_q(k) r_s[k ^ e_q] mu_s[k]   (to dL/dtheta_q, summed over s)
//   D_q = sum_k sign_q(k) r_0[k ^ e_q] mu_s[k]   (s >= 1: dL/dJ_{q, s-1})
// with sign_q(k) = +1 where qubit q is 1. r_s is a product over qubits: the five lowest index
// bits come from 32-entry tables, the higher ones from a per-chunk factor, so every sum splits
// into 32-column correlations. Four drain warps take a finished tile's correlations out of
// tensor memory while eight staging warps and the tensor core work on the next tile (the two
// accumulator buffers alternate).
struct MuArgs {
  const float* thetaJ;     // [P][n] float4
  const __half* WT16;      // FP16 pairs of 2^14 U' transposed, [2 dim / HKC][hi, lo][dim x HKC]
  const float* lam;        // costate rows, blocked layout [2 dim / 256][rtot][256]
  int64_t rtot;
  float* dthetaJ;          // [P][n] float4 (dL/dtheta, dL/dJ_x, dL/dJ_y, dL/dJ_t)
  int32_t n;
  int64_t npts[3], pt_base[3], tile_end[3];
  int32_t* status;
  const int32_t* scal;     // [2] float bits; [1] = max |lambda| (scale of the costate operand)
};

// float4 offset of K-chunk kc (KC costate components) from the start of a row's first block.
__device__ __forceinline__ int64_t mu_koff(const MuArgs& a, int kc) {
  return ((int64_t)(kc / (256 / KC)) * a.rtot * 256 + (kc % (256 / KC)) * KC) / 4;
}

// Two stages of (A: costate rows, W: transposed operand), FP16 pairs, HKC-wide K steps, then
// the epilogue's exchange buffer.
__host__ __device__ inline int mu_smem_bytes(int n) {
  return 2 * (2 * TM * HKC * 2 + 2 * (1 << n) * HKC * 2) + 256 + 2 * 4 * 32 * 8 * 4;
}

// Per-row state of a tile being drained.
struct MuRow {
  float Lo[32], Lod[32];          // low five qubits: value and tangent-s product tables
  float hc[3], hs[3], hj[3];      // high qubits (n - 5 <= 3): cos, sin of theta/2, J along s
  float C[8], D[8];
};

__device__ __forceinline__ void mu_row_setup(const MuArgs& a, int n, int set, int64_t p, int s, MuRow& R) {
  const float4* tj = reinterpret_cast<const float4*>(a.thetaJ) + (a.pt_base[set] + p) * n;
#pragma unroll
  for (int t = 0; t < 32; ++t) { R.Lo[t] = 1.f; R.Lod[t] = 0.f; }
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const float4 tq = __ldg(tj + (n - 1 - b));
    float sn, cs;
    sincosf(0.5f * tq.x, &sn, &cs);
    const float J = s == 0 ? 0.f : (s == 1 ? tq.y : (s == 2 ? tq.z : tq.w));
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const bool bit = (t >> b) & 1;
      const float f = bit ? sn : cs, d = bit ? 0.5f * cs : -0.5f * sn;
      R.Lod[t] = R.Lod[t] * f + R.Lo[t] * d * J;
      R.Lo[t] *= f;
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    R.hc[q] = 1.f; R.hs[q] = 0.f; R.hj[q] = 0.f;
    if (q < n - 5) {
      const float4 tq = __ldg(tj + q);
      sincosf(0.5f * tq.x, &R.hs[q], &R.hc[q]);
      R.hj[q] = s == 0 ? 0.f : (s == 1 ? tq.y : (s == 2 ? tq.z : tq.w));
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) { R.C[q] = 0.f; R.D[q] = 0.f; }
}

// High-qubit factor of chunk index c (bits of k above the low five) and its tangent.
__device__ __forceinline__ void mu_high(const MuRow& R, int n, int c, float& H, float& Hd) {
  H = 1.f;
  Hd = 0.f;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < n - 5) {
      const bool bit = (c >> (n - 6 - q)) & 1;
      const float f = bit ? R.hs[q] : R.hc[q], d = bit ? 0.5f * R.hc[q] : -0.5f * R.hs[q];
      Hd = Hd * f + H * d * R.hj[q];
      H *= f;
    }
  }
}

// One 32-column chunk c of the row's mu (tensor memory) into C and D.
__device__ __forceinline__ void mu_chunk(MuRow& R, int n, int s, int c, uint32_t taddr, float us) {
  float v[32];   // scaled mu: the scale comes out of the correlations below
  qptc::tmem_ld32(taddr, v);
  float X = 0.f, Y = 0.f, A[5], B[5];
#pragma unroll
  for (int b = 0; b < 5; ++b) { A[b] = 0.f; B[b] = 0.f; }
#pragma unroll
  for (int l = 0; l < 32; ++l) {
    X += v[l] * R.Lo[l];
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const float sv = ((l >> b) & 1) ? v[l] : -v[l];
      A[b] += sv * R.Lo[l ^ (1 << b)];
    }
  }
  if (s != 0) {
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      Y += v[l] * R.Lod[l];
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        const float sv = ((l >> b) & 1) ? v[l] : -v[l];
        B[b] += sv * R.Lod[l ^ (1 << b)];
      }
    }
  }
  X *= us;
  Y *= us;
#pragma unroll
  for (int b = 0; b < 5; ++b) { A[b] *= us; B[b] *= us; }
  float H, Hd;
  mu_high(R, n, c, H, Hd);
  // low qubits q = n - 1 - b: the flip stays inside the chunk
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const int q = n - 1 - b;
#pragma unroll
    for (int qq = 0; qq < 8; ++qq) {
      if (qq == q) {
        R.C[qq] += s == 0 ? H * A[b] : Hd * A[b] + H * B[b];
        R.D[qq] += H * A[b];
      }
    }
  }
  // high qubits: the flip moves to chunk c ^ e
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < n - 5) {
      const int e = 1 << (n - 6 - q);
      float Hf, Hdf;
      mu_high(R, n, c ^ e, Hf, Hdf);
      const float sg = (c & e) ? 1.f : -1.f;
      R.C[q] += sg * (s == 0 ? Hf * X : Hdf * X + Hf * Y);
      R.D[q] += sg * Hf * X;
    }
  }
}

constexpr int MU_STAGERS = 256;   // operand staging (8 warps: two per row quarter, half a K step each)
constexpr int MU_DRAINERS = 128;  // embedding epilogue of the previous tile (4 warps, same rows)
constexpr int MU_THREADS = MU_STAGERS + MU_DRAINERS + 32;

// NQ = n (7 or 8, equal to a.n): the qubit count fixes the table bit positions and the qubit
// index of every correlation at compile time.
template <int NQ>
__global__ void __launch_bounds__(MU_THREADS, 1) dense_mu_embed_kernel(MuArgs a) {
  static_assert(NQ == 7 || NQ == 8, "one 256-column chunk of mu per row");
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int n = NQ, dim = 1 << n;
  constexpr int ktot = 2 * dim, nch = dim, nkc = ktot / HKC;   // dim <= 256: one column chunk
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool ctrl = warp == (MU_STAGERS + MU_DRAINERS) / 32;
  const int abytes = TM * HKC * 2, wbytes = nch * HKC * 2;
  // FP16 pairs: the costates scaled by one power of two from the recorded maximum, the
  // operand blocks by 2^14; both come back out in the drain
  const float sL = pow2_scale(__int_as_float(__ldg(a.scal + 1)));
  const float us = 1.f / (sL * W16_SCALE);
  const int stage_bytes = 2 * abytes + 2 * wbytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);
  uint64_t* w_full = bars;         // [2] W operand of a stage landed
  uint64_t* mma_done = bars + 2;   // [2] tensor-core work of a stage finished
  uint64_t* a_full = bars + 4;     // [2] A operand of a stage written (8 staging warps)
  uint64_t* acc_free = bars + 6;   // [2] a tensor-memory buffer drained (4 drain warps)
  uint64_t* tile_done = bars + 8;  // [2] all MMAs of the tile in a tensor-memory buffer finished
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage_bytes + 96);
  float* ex = reinterpret_cast<float*>(sm + 2 * stage_bytes + 128);    // [2 (C, D)][4][32][8]
  const uint32_t tcols = 2 * nch <= 256 ? (2 * nch <= 128 ? 128 : 256) : 512;
  if (warp == 0) qptc::tmem_alloc(tslot, tcols);
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) qptc::mbar_init(&bars[i], 1);
    for (int i = 4; i < 6; ++i) qptc::mbar_init(&bars[i], MU_STAGERS / 32);
    for (int i = 6; i < 8; ++i) qptc::mbar_init(&bars[i], MU_DRAINERS / 32);
    for (int i = 8; i < 10; ++i) qptc::mbar_init(&bars[i], 1);
  }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const int nchunk32 = dim / 32;
  const int64_t T2 = a.tile_end[2];
  bool ok = true;
  if (ctrl) {
    // ---- control thread: W copies one step ahead, MMAs as soon as a stage's A is written
    if (lane == 0) {
      const uint32_t id = qptc::idesc(0, TM, nch);
      const int64_t ntl = (int64_t)blockIdx.x < T2 ? (T2 - 1 - blockIdx.x) / gridDim.x + 1 : 0;
      const int64_t total = ntl * nkc;
      int64_t last_copy = -1, last_commit = -1;
      uint32_t it = 0;
      if (total > 0) {
        qptc::mbar_arrive_expect_tx(&w_full[0], 2 * wbytes);
        qptc::bulk_g2s(sm + 2 * abytes, a.WT16, 2 * wbytes, &w_full[0]);
        last_copy = 0;
      }
      for (int64_t t = 0; t < ntl && ok; ++t) {
        const uint32_t buf = t & 1;
        // the buffer's previous tile (t - 2) must be drained before it is overwritten
        if (t >= 2) ok = qptc::mbar_wait(&acc_free[buf], (uint32_t)((t - 2) >> 1) & 1);
        for (int kc = 0; kc < nkc && ok; ++kc, ++it) {
          const uint32_t st = it & 1;
          ok = qptc::mbar_wait(&w_full[st], (it >> 1) & 1);
          if (ok) ok = qptc::mbar_wait(&a_full[st], (it >> 1) & 1);
          if (!ok) break;
          qptc::fence_after();
          const uint32_t sa = qptc::smem_u32(sm + st * stage_bytes), sw = sa + 2 * abytes;
          const uint32_t dt = tmem + buf * (tcols / 2);
#pragma unroll
          for (int ks = 0; ks < HKC / 16; ++ks) {
            const uint64_t ah = qptc::desc_kmajor(sa + ks * 256, 128, (HKC / 8) * 128);
            const uint64_t al = qptc::desc_kmajor(sa + abytes + ks * 256, 128, (HKC / 8) * 128);
            const uint64_t wh = qptc::desc_kmajor(sw + ks * 256, 128, (HKC / 8) * 128);
            const uint64_t wl = qptc::desc_kmajor(sw + wbytes + ks * 256, 128, (HKC / 8) * 128);
            qptc::mma_f16(dt, ah, wh, id, (kc > 0 || ks > 0) ? 1u : 0u);
            qptc::mma_f16(dt, ah, wl, id, 1u);
            qptc::mma_f16(dt, al, wh, id, 1u);
          }
          qptc::commit(&mma_done[st]);
          if (kc == nkc - 1) qptc::commit(&tile_done[buf]);   // the drain warps may read it
          last_commit = it;
          if ((int64_t)it + 1 < total) {
            const uint32_t s2 = (it + 1) & 1;
            if (it >= 1) ok = qptc::mbar_wait(&mma_done[s2], ((it - 1) >> 1) & 1);
            if (!ok) break;
            qptc::mbar_arrive_expect_tx(&w_full[s2], 2 * wbytes);
            qptc::bulk_g2s(sm + s2 * stage_bytes + 2 * abytes, a.WT16 + (int64_t)((kc + 1) % nkc) * 2 * (nch * HKC),
                           2 * wbytes, &w_full[s2]);
            last_copy = it + 1;
          }
        }
      }
      if (!ok) {
        atomicExch(a.status, 6);
        if (last_copy >= 0) qptc::mbar_wait(&w_full[last_copy & 1], ((uint32_t)last_copy >> 1) & 1);
        if (last_commit >= 0) qptc::mbar_wait(&mma_done[last_commit & 1], ((uint32_t)last_commit >> 1) & 1);
      }
    }
  } else if (warp < MU_STAGERS / 32) {
    // ---- staging warps: costate rows -> FP16-pair A operand; warps w and w + 4 share the rows
    // of quarter w, each splitting half of a K step's 32 components
    const int rw = warp & 3, kh = warp >> 2;
    const int row = rw * 32 + lane;
    uint32_t it = 0;
    // costate row of this thread in a tile (A operand source)
    auto tile_row = [&](int64_t tile) -> const float4* {
      int set;
      int64_t p0;
      if (tile < a.tile_end[0]) { set = 0; p0 = tile * 32; }
      else if (tile < a.tile_end[1]) { set = 1; p0 = (tile - a.tile_end[0]) * TM; }
      else { set = 2; p0 = (tile - a.tile_end[1]) * TM; }
      const int64_t np = a.npts[set];
      const int64_t p = p0 + (set == 0 ? lane : row);
      const int64_t pc = p < np ? p : np - 1;
      return reinterpret_cast<const float4*>(a.lam + lam_row(set, pc, set == 0 ? rw : 0, a.npts[0], a.pt_base[set]) * 256) +
             kh * (KC / 8);
    };
    // the next K-step's four float4 of this thread's half row are loaded one step ahead
    float4 nxt[KC / 8];
    if ((int64_t)blockIdx.x < T2) {
      const float4* s0 = tile_row(blockIdx.x);
#pragma unroll
      for (int g4 = 0; g4 < KC / 8; ++g4) nxt[g4] = __ldg(s0 + g4);
    }
    for (int64_t tile = blockIdx.x; tile < T2 && ok; tile += gridDim.x) {
      const float4* src = tile_row(tile);
      const float4* src_next = tile + gridDim.x < T2 ? tile_row(tile + gridDim.x) : nullptr;
      for (int kc = 0; kc < nkc; ++kc, ++it) {
        const uint32_t st = it & 1;
        unsigned char* sA = sm + st * stage_bytes;
        if (it >= 2 && ok) ok = qptc::mbar_wait(&mma_done[st], ((it - 2) >> 1) & 1);
        float4 cur[KC / 8];
#pragma unroll
        for (int g4 = 0; g4 < KC / 8; ++g4) cur[g4] = nxt[g4];
        const float4* ns = kc + 1 < nkc ? src + mu_koff(a, kc + 1) : src_next;
        if (ns) {
#pragma unroll
          for (int g4 = 0; g4 < KC / 8; ++g4) nxt[g4] = __ldg(ns + g4);
        }
        if (ok) {
#pragma unroll
          for (int g8 = 0; g8 < HKC / 16; ++g8) {
            const float v8[8] = {cur[2 * g8].x, cur[2 * g8].y, cur[2 * g8].z, cur[2 * g8].w,
                                 cur[2 * g8 + 1].x, cur[2 * g8 + 1].y, cur[2 * g8 + 1].z, cur[2 * g8 + 1].w};
            uint4 h8, l8;
            pack_h8(v8, sL, h8, l8);
            const uint32_t off = core_off_h(row, kh * (HKC / 2) + g8 * 8);
            *reinterpret_cast<uint4*>(sA + off) = h8;
            *reinterpret_cast<uint4*>(sA + abytes + off) = l8;
          }
        }
        qptc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) qptc::mbar_arrive(&a_full[st]);
      }
      ok = qptc::bar_and(1, MU_STAGERS, ok);
    }
    if (!ok && lane == 0) atomicExch(a.status, 6);
  } else {
    // ---- drain warps: the embedding correlations of each finished tile, read from tensor
    // memory while the staging warps and the tensor core work on the next tile (drain warp w
    // reads tensor-memory lane quarter w, the rows that staging warps w and w + 4 wrote)
    const int dw = warp - MU_STAGERS / 32;
    MuRow R;
    auto bar = [&]() {
      __syncwarp();   // bar.sync is the aligned form
      asm volatile("bar.sync 2, %0;" ::"r"(MU_DRAINERS) : "memory");
    };
    uint32_t t = 0;
    for (int64_t tile = blockIdx.x; tile < T2 && ok; tile += gridDim.x, ++t) {
      int set;
      int64_t p0;
      if (tile < a.tile_end[0]) { set = 0; p0 = tile * 32; }
      else if (tile < a.tile_end[1]) { set = 1; p0 = (tile - a.tile_end[0]) * TM; }
      else { set = 2; p0 = (tile - a.tile_end[1]) * TM; }
      const bool nv4 = set == 0;
      const int64_t np = a.npts[set];
      const int64_t p = p0 + (nv4 ? lane : dw * 32 + lane);
      const int s = nv4 ? dw : 0;
      const uint32_t buf = t & 1;
      ok = qptc::bar_and(2, MU_DRAINERS, ok && qptc::mbar_wait(&tile_done[buf], (t >> 1) & 1));
      if (!ok) break;
      qptc::fence_after();
      mu_row_setup(a, n, set, p < np ? p : np - 1, s, R);
      for (int c = 0; c < nchunk32; ++c)
        mu_chunk(R, n, s, c, tmem + ((uint32_t)(dw * 32) << 16) + buf * (tcols / 2) + c * 32, us);
      qptc::fence_before();
      // rows of one point sit in four warps (same lane): combine through shared memory
      if (nv4) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          ex[(s * 32 + lane) * 8 + q] = R.C[q];
          ex[1024 + (s * 32 + lane) * 8 + q] = R.D[q];
        }
      }
      bar();
      if (p < np && (!nv4 || dw == 0)) {
        float4* dst = reinterpret_cast<float4*>(a.dthetaJ) + (a.pt_base[set] + p) * n;
        for (int q = 0; q < n; ++q) {
          if (nv4) {
            const float c = ex[lane * 8 + q] + ex[(32 + lane) * 8 + q] + ex[(64 + lane) * 8 + q] + ex[(96 + lane) * 8 + q];
            dst[q] = make_float4(c, ex[1024 + (32 + lane) * 8 + q], ex[1024 + (64 + lane) * 8 + q],
                                 ex[1024 + (96 + lane) * 8 + q]);
          } else {
            float c = 0.f;
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) if (qq == q) c = R.C[qq];
            dst[q] = make_float4(c, 0.f, 0.f, 0.f);
          }
        }
      }
      bar();
      // the buffer is fully read: the control thread may overwrite it
      if (lane == 0) qptc::mbar_arrive(&acc_free[buf]);
    }
    if (!ok && lane == 0) atomicExch(a.status, 6);
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, tcols);
}

}  // namespace qpd
