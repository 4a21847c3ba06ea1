// qp_dense.cuh -- fused-unitary path: the input-independent ansatz layers are multiplied into
// one 2^n x 2^n unitary U, and the PQC state of every point (and its three tangents) is
// U applied to the embedded product state, computed as one dense contraction on the
// 5th-generation tensor cores.
//
// With the RX embedding, G(theta)|0> = (cos theta/2, -i sin theta/2): every amplitude of the
// product state and of its tangents is a real number times the phase (-i)^{popcount k}
// (identity phase for RY). Folding that phase into the columns, U' = U D, leaves a real
// operand R (one row per point and vector):
//   Phi^T[(point, s), (amp j, re|im)] = sum_k R_s[k] W[(j, re|im), k],  W = [Re U'; Im U'].
// R is generated in shared memory from the per-point angles (never stored in HBM); W is
// streamed by bulk copies; the product runs in 3xTF32 (hi*hi + hi*lo + lo*hi, FP32
// accumulation in tensor memory).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "qp_aux.cuh"
#include "qp_circuit.cuh"
#include "qp_common.h"
#include "qp_tc.cuh"

namespace qpd {

constexpr int KC = 32;        // K (basis index) elements per chunk
constexpr int TM = 128;       // rows per tile (tensor-memory lanes)

// Output columns per chunk of the 3xTF32 row contractions (at most 128: two accumulators of
// a chunk, double-buffered, fill the 512 tensor-memory columns).
__host__ __device__ inline int n_cols_chunk(int n) { return (2 << n) < 128 ? (2 << n) : 128; }

// Byte offset of element (row r, k-in-chunk t) in a K-major, no-swizzle operand block whose
// 8-row groups hold KC/4 core matrices of 8 x 16 bytes.
__host__ __device__ inline uint32_t core_off(int r, int t) {
  return (uint32_t)((r >> 3) * (KC / 4) * 128 + (t >> 2) * 128 + (r & 7) * 16 + (t & 3) * 4);
}

constexpr int FKC = 16;       // K per pipeline stage of the weight-gradient kernel (TF32)
constexpr int HKC = 32;       // K per pipeline stage of the fused forward kernel (FP16 pairs)
// Fixed power-of-two scale of the fused unitary's FP16 operand pair (|U'| <= 1).
constexpr float W16_SCALE = 16384.f;
// The same layout with 16-element K chunks (operand blocks of the fused forward kernel).
__host__ __device__ inline uint32_t core_off16(int r, int t) {
  return (uint32_t)((r >> 3) * (FKC / 4) * 128 + (t >> 2) * 128 + (r & 7) * 16 + (t & 3) * 4);
}
// Byte offset of 16-bit element (row r, K index k) in a K-major HKC-wide block: core matrices
// of 8 rows x 8 elements, K-adjacent ones 128 bytes apart, 8-row groups (HKC / 8) * 128 apart.
__host__ __device__ inline uint32_t core_off_h(int r, int k) {
  return (uint32_t)((r >> 3) * (HKC / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Power-of-two scale that puts magnitudes up to `mx` below 2^13 (1 when mx is not positive).
__device__ __forceinline__ float pow2_scale(float mx) {
  if (!(mx > 0.f)) return 1.f;
  int e = 0;
  frexpf(mx, &e);
  return ldexpf(1.f, max(-100, min(100, 13 - e)));
}
// Eight scaled values as FP16 pairs (hi, lo = rounding remainder), packed for one 16-byte store.
__device__ __forceinline__ void pack_h8(const float* v, float sc, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float x0 = sc * v[2 * e], x1 = sc * v[2 * e + 1];
    const __half2 h2 = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h2);
    const __half2 l2 = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    h[e] = *reinterpret_cast<const uint32_t*>(&h2);
    l[e] = *reinterpret_cast<const uint32_t*>(&l2);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Blocked costate layout of the fused path (n = 7, 8): [2^(n+1) / 256][rows][256] floats, rows
// = 4 per collocation point (vector-major inside the point), then the IC and BC points with
// one row each. A 16-row step of the weight-gradient contraction is one contiguous 16 KiB run
// per 256-column block.
__host__ __device__ inline int64_t lam_row(int set, int64_t p, int s, int64_t n0, int64_t base) {
  return set == 0 ? p * 4 + s : 3 * n0 + base + p;
}

// cos and sin of theta / 2 for every (point, qubit) angle, once per call (the encoding factors
// of the product states, shared by the contractions that regenerate them).
__global__ void dense_halfangle_kernel(const float4* thetaJ, float2* cs, int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    float sn, c;
    sincosf(0.5f * thetaJ[i].x, &sn, &c);
    cs[i] = make_float2(c, sn);
  }
}

// ------------------------------------------------------------------------- unitary build
struct BuildArgs {
  const float* params;
  int64_t circ_off;
  int32_t n, L, ansatz, enc;
  float* W;        // [ncc][nkc][2 (hi, lo)][nch x KC] tiled operand blocks
  double2* U;      // [2^n][2^n] fused unitary U' (row j, column k), FP64, or null
  float* WT;       // transpose operand (rows a = basis index, K = o), same tiling, or null
  __half* W16;     // [dim / HKC][2 dim / 256][2 (hi, lo)][256 x HKC] FP16 pairs of W * W16_SCALE, or null
  double2* gates;  // [L][n][4] rotation gate matrices (written by block 0), or null
  const double2* crz64;  // CRZ mesh ansatze: [L][2^n] diagonal (cos, sin) of each layer's mesh
  __half* WT16;    // [2 dim / HKC][hi, lo][dim x HKC] FP16 pairs of 2^14 U' transposed (mu kernel), or null
};

__device__ inline double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Single-qubit gate of (layer l, qubit q) in double precision (same formulas as the build).
__device__ inline void gate_fp64(const float* params, int64_t circ_off, int ansatz, int n, int l, int q,
                                 double2* g) {
  const int kp = qp_ansatz_k(ansatz);
  const float* p = params + circ_off + (int64_t)l * qp_layer_params(ansatz, n) + (int64_t)q * kp;
  if (ansatz == 4 || ansatz == 5) {
    // RX(a), then RZ(b) for the two-rotation Cross-Mesh: RZ multiplies row 0 by e^{-ib/2} and
    // row 1 by e^{ib/2}
    double c, sn, cb = 1.0, sb = 0.0;
    sincos(0.5 * (double)p[0], &sn, &c);
    if (ansatz == 5) sincos(0.5 * (double)p[1], &sb, &cb);
    g[0] = make_double2(cb * c, -sb * c); g[1] = make_double2(-sn * sb, -sn * cb);
    g[2] = make_double2(sn * sb, -sn * cb); g[3] = make_double2(cb * c, sb * c);
  } else if (ansatz == 0) {
    double ca, sa, cb, sb;
    sincos(0.5 * (double)p[0], &sa, &ca);
    sincos(0.5 * (double)p[1], &sb, &cb);
    g[0] = make_double2(cb * ca, -sb * ca); g[1] = make_double2(-cb * sa, sb * sa);
    g[2] = make_double2(cb * sa, sb * sa); g[3] = make_double2(cb * ca, sb * ca);
  } else {
    double cb, sb;
    sincos(0.5 * (double)p[1], &sb, &cb);
    const double ap = 0.5 * ((double)p[0] + (double)p[2]), am = 0.5 * ((double)p[0] - (double)p[2]);
    double cp, sp, cm, smm;
    sincos(ap, &sp, &cp);
    sincos(am, &smm, &cm);
    g[0] = make_double2(cp * cb, -sp * cb); g[1] = make_double2(-cm * sb, -smm * sb);
    g[2] = make_double2(cm * sb, -smm * sb); g[3] = make_double2(cp * cb, sp * cb);
  }
}

// Index map of the CNOTs of layer l (ring or mesh; basis state |k> -> |c(k)>).
__device__ __forceinline__ int ring_map(int n, int ansatz, int l, int k) {
  return (int)qp_ent_map(n, ansatz, l, (uint32_t)k);
}

// Gate matrices of every (layer, qubit) in FP64, once per call (one thread each).
__global__ void dense_gates_kernel(BuildArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.L * a.n) gate_fp64(a.params, a.circ_off, a.ansatz, a.n, i / a.n, i % a.n, &a.gates[i * 4]);
}

// Double-float arithmetic (an unevaluated sum h + l of two floats, ~48-bit significand): the
// build runs on the FP32 pipes, which on this part are 64x the FP64 rate. Products by the
// exact FMA residual, sums by the two-sum of Knuth with the low parts added.
struct DFl {
  float h, l;
};
__device__ __forceinline__ DFl df_mul(float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  return {p, e};
}
__device__ __forceinline__ DFl df_add(DFl a, DFl b) {
  const float s = a.h + b.h, bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb) + a.l + b.l;
  const float h = s + e;
  return {h, e - (h - s)};
}
// (g x) for a double-float complex g = (re h, re l, im h, im l) and amplitude x, same layout:
// the real and imaginary parts as 2-term dot products.
__device__ __forceinline__ void df_cmac(const float4& g, const float4& x, DFl& re, DFl& im) {
  re = df_add(df_mul(g.x, g.y, x.x, x.y), df_mul(-g.z, -g.w, x.z, x.w));
  im = df_add(df_mul(g.x, g.y, x.z, x.w), df_mul(g.z, g.w, x.x, x.y));
}
__device__ __forceinline__ float4 df_split(double v0, double v1) {
  const float h0 = (float)v0, h1 = (float)v1;
  return make_float4(h0, (float)(v0 - (double)h0), h1, (float)(v1 - (double)h1));
}

// One block per basis column k: |k> through all layers (gates and CNOT rings) in double-float
// arithmetic from the FP64 gate matrices. A gate is one pass over the amplitude pairs, a CNOT
// ring one permutation pass.
__global__ void dense_build_kernel(BuildArgs a) {
  extern __shared__ __align__(16) float4 colbuf[];  // two [2^n] column buffers (double-float complex)
  __shared__ float4 gm[QP_MAXL * QP_MAXQ * 4];
  const int n = a.n, dim = 1 << n, k = blockIdx.x;
  for (int i = threadIdx.x; i < a.L * n * 4; i += blockDim.x) {
    const double2 g = a.gates[i];
    gm[i] = df_split(g.x, g.y);
  }
  float4* col = colbuf;
  float4* nxt = colbuf + dim;
  for (int j = threadIdx.x; j < dim; j += blockDim.x) col[j] = make_float4(j == k ? 1.f : 0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  for (int l = 0; l < a.L; ++l) {
    for (int q = 0; q < n; ++q) {
      const float4* g = &gm[(l * n + q) * 4];
      const int bit = 1 << (n - 1 - q);
      for (int i = threadIdx.x; i < dim / 2; i += blockDim.x) {
        const int k0 = ((i & ~(bit - 1)) << 1) | (i & (bit - 1));
        const int k1 = k0 | bit;
        const float4 x = col[k0], y = col[k1];
        DFl r0, i0, r1, i1, r2, i2, r3, i3;
        df_cmac(g[0], x, r0, i0);
        df_cmac(g[1], y, r1, i1);
        df_cmac(g[2], x, r2, i2);
        df_cmac(g[3], y, r3, i3);
        const DFl ar = df_add(r0, r1), ai = df_add(i0, i1), br = df_add(r2, r3), bi = df_add(i2, i3);
        col[k0] = make_float4(ar.h, ar.l, ai.h, ai.l);
        col[k1] = make_float4(br.h, br.l, bi.h, bi.l);
      }
      __syncthreads();
    }
    if (qp_has_crz(a.ansatz)) {
      // CRZ mesh: one phase per basis index
      for (int j = threadIdx.x; j < dim; j += blockDim.x) {
        const double2 d = a.crz64[(int64_t)l * dim + j];
        const float4 x = col[j];
        DFl re, im;
        df_cmac(df_split(d.x, d.y), x, re, im);
        col[j] = make_float4(re.h, re.l, im.h, im.l);
      }
      __syncthreads();
    } else if (a.ansatz != 3 && n > 1) {
      for (int j = threadIdx.x; j < dim; j += blockDim.x) nxt[ring_map(n, a.ansatz, l, j)] = col[j];
      __syncthreads();
      float4* t = col;
      col = nxt;
      nxt = t;
    }
  }
  // fold the embedding phase (-i)^{popcount k} (RX) into column k
  double2 ph = make_double2(1.0, 0.0);
  if (a.enc == 0) {
    const int m = __popc(k) & 3;
    ph = m == 0 ? make_double2(1, 0) : m == 1 ? make_double2(0, -1) : m == 2 ? make_double2(-1, 0) : make_double2(0, 1);
  }
  const int nch = n_cols_chunk(n), nkc = dim / KC;
  const int kc = k / KC, t = k % KC;
  for (int j = threadIdx.x; j < dim; j += blockDim.x) {
    const float4 cj = col[j];
    const double2 v = zmul(make_double2((double)cj.x + (double)cj.y, (double)cj.z + (double)cj.w), ph);
    if (a.U) a.U[(int64_t)j * dim + k] = v;
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      const int o = 2 * j + c2;
      const float x = (float)(c2 == 0 ? v.x : v.y);
      float hi, lo;
      {
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
        hi = __uint_as_float(h);
        uint32_t l2;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l2) : "f"((float)((c2 == 0 ? v.x : v.y) - (double)hi)));
        lo = __uint_as_float(l2);
      }
      if (a.W) {
        const int c = o / nch, r = o % nch;
        float* blk = a.W + ((int64_t)(c * nkc + kc) * 2) * (nch * KC);
        blk[core_off(r, t) / 4] = hi;
        blk[nch * KC + core_off(r, t) / 4] = lo;
      }
      if (a.W16) {
        // FP16 pair of the scaled element: x = hi + lo to about 2^-24 relative
        const int nc16 = (2 * dim) / 256, c = o / 256, r = o % 256;
        const double xs = (c2 == 0 ? v.x : v.y) * (double)W16_SCALE;
        const __half hh = __double2half(xs);
        const __half hl = __double2half(xs - (double)__half2float(hh));
        __half* blk = a.W16 + ((int64_t)((k / HKC) * nc16 + c) * 2) * (256 * HKC);
        blk[core_off_h(r, k % HKC) / 2] = hh;
        blk[256 * HKC + core_off_h(r, k % HKC) / 2] = hl;
      }
      if (a.WT16) {
        // transposed FP16 pairs: row a = k (N = dim <= 256), K = o in HKC-wide steps
        const double xs = (c2 == 0 ? v.x : v.y) * (double)W16_SCALE;
        const __half hh = __double2half(xs);
        const __half hl = __double2half(xs - (double)__half2float(hh));
        __half* blk = a.WT16 + (int64_t)(o / HKC) * 2 * (dim * HKC);
        blk[core_off_h(k, o % HKC) / 2] = hh;
        blk[dim * HKC + core_off_h(k, o % HKC) / 2] = hl;
      }
      if (a.WT) {
        // transpose: row a = k (N = dim, chunks of nch2), K = o (2 dim, chunks of KC)
        const int nch2 = dim < 128 ? dim : 128, nkc2 = 2 * dim / KC;
        const int c2b = k / nch2, r2 = k % nch2, kc2 = o / KC, t2 = o % KC;
        float* blk2 = a.WT + ((int64_t)(c2b * nkc2 + kc2) * 2) * (nch2 * KC);
        blk2[core_off(r2, t2) / 4] = hi;
        blk2[nch2 * KC + core_off(r2, t2) / 4] = lo;
      }
    }
  }
}

// ------------------------------------------------------------------------- forward GEMM
struct GemmArgs {
  const float* thetaJ;      // [P][n] float4 (theta, dtheta/dx, dtheta/dy, dtheta/dt)
  const float* W;
  float2* phi;              // [P][4][2^n] complex amplitudes
  int32_t n, nv;            // nv = 4 (state + tangents) or 1
  int64_t npts, pt_base;    // points of this set, first global point row
  int32_t* status;
  const float* lam;         // MODE 1: costate rows [P][4][2 dim] (A operand)
  float* mu;                // MODE 1: output rows [P][4][dim]
  const float2* cs;         // [P][n] (cos, sin) of theta / 2, or null (computed from thetaJ)
};

// Output columns per chunk for the two modes: MODE 0 (forward) has 2 dim outputs over K = dim;
// MODE 1 (back-projection mu = Re(U'^H lambda)) has dim outputs over K = 2 dim.
__host__ __device__ inline int row_nch(int n, int mode) {
  const int ntot = mode == 0 ? (2 << n) : (1 << n);
  return ntot < 128 ? ntot : 128;
}
// Smem: 2 stages x (A hi, A lo: 128 x KC fp32; W hi, W lo: nch x KC fp32) + barriers.
__host__ __device__ inline int gemm_smem_bytes(int n, int mode = 0) {
  const int nch = row_nch(n, mode);
  return 2 * (2 * TM * KC * 4 + 2 * nch * KC * 4) + 128;
}

// Row GEMM over (point, vector) rows on 3xTF32 operands. MODE 0: Phi = R W^T with R generated
// from the angles. MODE 1: mu = Lambda W (rows of Lambda loaded, B operand the transposed
// blocks). The tensor core adds each instruction's products into the FP32 accumulator with a
// truncating alignment (about one accumulator ulp per instruction, not averaging out over K),
// so the hi*hi products go to one accumulator and the hi*lo + lo*hi corrections, 2^-11
// smaller, to a second: K / 8 truncations on the result instead of 3K / 8. Each column chunk
// (at most 128 columns) therefore takes 2 x nch columns, double-buffered across chunks.
template <int MODE>
__global__ void __launch_bounds__(128, 1) dense_row_gemm_kernel(GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int n = a.n, dim = 1 << n;
  const int ktot = MODE == 0 ? dim : 2 * dim, ntot = MODE == 0 ? 2 * dim : dim;
  const int nch = row_nch(n, MODE), ncc = ntot / nch, nkc = ktot / KC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int abytes = TM * KC * 4, wbytes = nch * KC * 4;
  const int stage_bytes = 2 * abytes + 2 * wbytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);  // w_full[2], mma_done[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage_bytes + 64);
  // two buffers x (hi*hi accumulator, correction accumulator) of nch columns each
  const uint32_t tcols = nch * 4 <= 32 ? 32 : (nch * 4 <= 64 ? 64 : (nch * 4 <= 128 ? 128 : (nch * 4 <= 256 ? 256 : 512)));
  if (warp == 0) qptc::tmem_alloc(tslot, tcols);
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) qptc::mbar_init(&bars[i], 1);
  }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = qptc::idesc(2, TM, nch);

  // rows of a tile: nv = 4 -> 32 points x 4 vectors (warp = vector), nv = 1 -> 128 points
  const int ppt = TM / a.nv;
  const int64_t ntiles = (a.npts + ppt - 1) / ppt;
  const int s = a.nv == 4 ? warp : 0;
  const int prow = a.nv == 4 ? lane : tid;
  const int low = n < 5 ? n : 5;  // qubits n-low .. n-1 are the low index bits of a chunk
  bool ok = true;
  uint32_t it = 0;      // global item counter (stage = it & 1)
  int pending = -1;     // column chunk whose epilogue is pending (buffer = pend_buf)
  int64_t pend_tile = 0;
  uint32_t pend_buf = 0, pend_it = 0;
  uint32_t cbuf = 0;    // accumulator buffer of the current column chunk
  float Lo[32], Lod[32];

  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t p = tile * ppt + prow;
    const bool active = p < a.npts;
    const int64_t pc = active ? p : a.npts - 1;
    const float4* tj = reinterpret_cast<const float4*>(a.thetaJ) + (a.pt_base + pc) * n;
    // low-bit tables: Lo[t] = prod over the low qubits, Lod[t] its derivative along v_{s-1}
#pragma unroll
    for (int t = 0; t < 32; ++t) { Lo[t] = 1.f; Lod[t] = 0.f; }
    for (int b = 0; b < (MODE == 0 ? low : 0); ++b) {
      const int q = n - 1 - b;
      const float4 tq = tj[q];
      float sn, cs;
      sincosf(0.5f * tq.x, &sn, &cs);
      const float J = s == 1 ? tq.y : (s == 2 ? tq.z : tq.w);
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const bool bit = (t >> b) & 1;
        const float f = bit ? sn : cs, d = bit ? 0.5f * cs : -0.5f * sn;
        Lod[t] = Lod[t] * f + Lo[t] * d * J;
        Lo[t] *= f;
      }
    }
    for (int c = 0; c < ncc && ok; ++c) {
      for (int kc = 0; kc < nkc && ok; ++kc, ++it) {
        const uint32_t st = it & 1;
        unsigned char* sA = sm + st * stage_bytes;
        unsigned char* sW = sA + 2 * abytes;
        bool w_ok = true;
        if (it >= 2) w_ok = qptc::mbar_wait(&bars[2 + st], ((it - 2) >> 1) & 1);
        ok = __syncthreads_and(w_ok);  // every thread takes the same branch
        if (!ok) break;
        if (tid == 0) {
          qptc::mbar_arrive_expect_tx(&bars[st], 2 * wbytes);
          qptc::bulk_g2s(sW, a.W + (int64_t)(c * nkc + kc) * 2 * (nch * KC), 2 * wbytes, &bars[st]);
          // (MODE 1 passes the transposed blocks in a.W)
        }
        float* Ahi = reinterpret_cast<float*>(sA);
        float* Alo = reinterpret_cast<float*>(sA + abytes);
        const int r = tid;  // tile row owned by this thread
        if (MODE == 1) {
          const float4* src = reinterpret_cast<const float4*>(a.lam + ((a.pt_base + pc) * 4 + s) * (int64_t)ktot +
                                                              kc * KC);
#pragma unroll
          for (int g4 = 0; g4 < KC / 4; ++g4) {
            const float4 v4 = src[g4];
            float4 h4, l4;
            qptc::split_tf32(v4.x, h4.x, l4.x);
            qptc::split_tf32(v4.y, h4.y, l4.y);
            qptc::split_tf32(v4.z, h4.z, l4.z);
            qptc::split_tf32(v4.w, h4.w, l4.w);
            const uint32_t off = core_off(r, g4 * 4) / 4;
            *reinterpret_cast<float4*>(Ahi + off) = h4;
            *reinterpret_cast<float4*>(Alo + off) = l4;
          }
        } else {
        // high-bit factor H and its derivative for this chunk (qubits 0 .. n-1-low)
        float H = 1.f, Hd = 0.f;
        for (int q = 0; q < n - low; ++q) {
          const float4 tq = tj[q];
          float sn, cs;
          sincosf(0.5f * tq.x, &sn, &cs);
          const bool bit = (kc >> (n - low - 1 - q)) & 1;
          const float f = bit ? sn : cs, d = bit ? 0.5f * cs : -0.5f * sn;
          const float J = s == 1 ? tq.y : (s == 2 ? tq.z : tq.w);
          Hd = Hd * f + H * d * J;
          H *= f;
        }
#pragma unroll
        for (int g4 = 0; g4 < KC / 4; ++g4) {
          float4 h4, l4;
          float* hv = &h4.x;
          float* lv = &l4.x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int t = g4 * 4 + e;
            const float v = s == 0 ? H * Lo[t] : Hd * Lo[t] + H * Lod[t];
            qptc::split_tf32(v, hv[e], lv[e]);
          }
          const uint32_t off = core_off(r, g4 * 4) / 4;
          *reinterpret_cast<float4*>(Ahi + off) = h4;
          *reinterpret_cast<float4*>(Alo + off) = l4;
        }
        }
        qptc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          ok = qptc::mbar_wait(&bars[st], (it >> 1) & 1);
          if (ok) {
            qptc::fence_after();
            const uint32_t sa = qptc::smem_u32(sA), sw = qptc::smem_u32(sW);
            const uint32_t dt = tmem + cbuf * (tcols / 2);   // hi*hi accumulator
            const uint32_t dc = dt + nch;                      // correction accumulator
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
              const uint64_t ah = qptc::desc_kmajor(sa + ks * 256, 128, (KC / 4) * 128);
              const uint64_t al = qptc::desc_kmajor(sa + abytes + ks * 256, 128, (KC / 4) * 128);
              const uint64_t wh = qptc::desc_kmajor(sw + ks * 256, 128, (KC / 4) * 128);
              const uint64_t wl = qptc::desc_kmajor(sw + wbytes + ks * 256, 128, (KC / 4) * 128);
              const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
              qptc::mma_tf32(dt, ah, wh, id, acc);
              qptc::mma_tf32(dc, ah, wl, id, acc);
              qptc::mma_tf32(dc, al, wh, id, 1u);
            }
            qptc::commit(&bars[2 + st]);
          }
        }
        ok = __syncthreads_and(ok);
        if (!ok) break;
        // drain the previous column chunk while this one runs on the tensor cores
        if (kc == 0 && pending >= 0) {
          ok = __syncthreads_and(qptc::mbar_wait(&bars[2 + (pend_it & 1)], (pend_it >> 1) & 1));
          if (ok) {
            qptc::fence_after();
            const int64_t pp = pend_tile * ppt + prow;
            float v[32], vc[32];
            for (int c0 = 0; c0 < nch; c0 += 32) {
              const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + pend_buf * (tcols / 2) + c0;
              qptc::tmem_ld32(ta, v);
              qptc::tmem_ld32(ta + nch, vc);
#pragma unroll
              for (int e = 0; e < 32; ++e) v[e] += vc[e];
              if (pp < a.npts) {
                float* orow = MODE == 0 ? reinterpret_cast<float*>(a.phi) : a.mu;
                float4* dst = reinterpret_cast<float4*>(orow + ((a.pt_base + pp) * 4 + s) * (int64_t)ntot +
                                                        pending * nch + c0);
#pragma unroll
                for (int e = 0; e < 8; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
              }
            }
            qptc::fence_before();
          }
          ok = __syncthreads_and(ok);
          pending = -1;
        }
        if (kc == nkc - 1) {
          pending = c;
          pend_tile = tile;
          pend_buf = cbuf;
          pend_it = it;
          cbuf ^= 1;
        }
      }
    }
  }
  if (ok && pending >= 0) {
    ok = __syncthreads_and(qptc::mbar_wait(&bars[2 + (pend_it & 1)], (pend_it >> 1) & 1));
    if (ok) {
      qptc::fence_after();
      const int64_t pp = pend_tile * ppt + prow;
      float v[32], vc[32];
      for (int c0 = 0; c0 < nch; c0 += 32) {
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + pend_buf * (tcols / 2) + c0;
        qptc::tmem_ld32(ta, v);
        qptc::tmem_ld32(ta + nch, vc);
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] += vc[e];
        if (pp < a.npts) {
          float* orow = MODE == 0 ? reinterpret_cast<float*>(a.phi) : a.mu;
          float4* dst = reinterpret_cast<float4*>(orow + ((a.pt_base + pp) * 4 + s) * (int64_t)ntot +
                                                  pending * nch + c0);
#pragma unroll
          for (int e = 0; e < 8; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
        }
      }
    }
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.status, 6);
    // let every tensor-core operation this CTA issued finish before freeing tensor memory
    if (it >= 1) qptc::mbar_wait(&bars[2 + ((it - 1) & 1)], ((it - 1) >> 1) & 1);
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------------------------------- row GEMMs, FP16 pairs
// Row contractions for n = 9, 10 (and the forward of qp_forward for n >= 7) on FP16 operand
// pairs, one 128-row tile of (point, vector) rows x 256 output columns at a time, K in
// 32-wide stages:
//   MODE 0, forward: Phi = R W^T, K = 2^n. W16 holds FP16 pairs of 2^14 W (the build); each
//     generated row of R is scaled by a power of two 2^(13-e) bounding it (|R_0| <= 1,
//     |R_d| <= sum_q |J_q,d| / 2). The largest bound goes to scal[0] (atomic maximum of the
//     float bits) for the weight gradient's operand scale.
//   MODE 1, back-projection: mu = Re(U'^H lambda) = Lambda W, K = 2^(n+1), N = 2^n. The B
//     operand is WT16 (FP16 pairs of 2^14 U'^T from the build); the costate rows are scaled by
//     one power of two from their largest magnitude, recorded by the pointwise stage.
// x = hi + lo to ~2^-22 for every operand.
//
// The tensor core adds each instruction's partial products into the FP32 accumulator with a
// truncating alignment, an error of up to one accumulator ulp per instruction that does not
// average out over K. The large hi*hi products therefore go to one accumulator and the small
// hi*lo + lo*hi corrections to a second (both 256 columns: the whole tensor memory), K / 16
// truncations instead of 3K / 16 on the result; the epilogue adds the two in FP32 and unscales.
//
// Warp roles: eight stager warps generate (MODE 0: two threads per row, one half of each
// 32-wide K stage) or load (MODE 1: coalesced, eight threads per row) the A operand, pack it
// into FP16 pairs and run the epilogue (warps w and w + 4 drain the two column halves of
// tensor-memory lanes 32 (w % 4) ..); a producer thread streams the B blocks by bulk copies as
// soon as a stage's tensor-core work is done; an MMA thread issues a stage's MMAs as soon as
// its A and B are in shared memory, so several stages of MMAs stay queued.
constexpr int F16_ST = 4;                            // pipeline stages
constexpr int F16_STAGERS = 256;                     // 8 stager warps
constexpr int F16_THREADS = F16_STAGERS + 64;        // + producer warp + MMA warp
constexpr int F16_ABYTES = TM * HKC * 2;             // one A half (hi or lo) of a stage
constexpr int F16_WBYTES = 256 * HKC * 2;            // one B half
constexpr int F16_STAGE = 2 * F16_ABYTES + 2 * F16_WBYTES;
__host__ __device__ inline int row16_smem_bytes() { return F16_ST * F16_STAGE + 128; }

// B operand block of iteration (column chunk c, K stage kc) into one stage (both halves).
template <int MODE>
__device__ __forceinline__ void row16_copy_b(const __half* B16, int dim, int ncc, int c, int kc, unsigned char* sW,
                                             uint64_t* bar) {
  qptc::mbar_arrive_expect_tx(bar, 2 * F16_WBYTES);
  if (MODE == 0) {
    // [K stage][column chunk][hi, lo][256 x HKC]
    qptc::bulk_g2s(sW, B16 + ((int64_t)kc * ncc + c) * 2 * (256 * HKC), 2 * F16_WBYTES, bar);
  } else {
    // [K stage][hi, lo][dim x HKC]: rows 256 c .. 256 c + 255 of each half
    const __half* blk = B16 + (int64_t)kc * 2 * (dim * HKC) + (int64_t)c * (256 * HKC);
    qptc::bulk_g2s(sW, blk, F16_WBYTES, bar);
    qptc::bulk_g2s(sW + F16_WBYTES, blk + (int64_t)dim * HKC, F16_WBYTES, bar);
  }
}

template <int MODE>
__global__ void __launch_bounds__(F16_THREADS, 1) dense_row16_kernel(GemmArgs a, const __half* B16, int32_t* scal) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int n = a.n, dim = 1 << n;
  const int ktot = MODE == 0 ? dim : 2 * dim, ntot = MODE == 0 ? 2 * dim : dim;
  const int ncc = ntot / 256, nkc = ktot / HKC, high = n - 5;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NSW = F16_STAGERS / 32;
  uint64_t* a_full = reinterpret_cast<uint64_t*>(sm + F16_ST * F16_STAGE);  // [ST] stager warps
  uint64_t* w_full = a_full + F16_ST;                                         // [ST] bulk copies
  uint64_t* mma_done = w_full + F16_ST;                                       // [ST] commit
  uint64_t* acc_full = mma_done + F16_ST;                                     // chunk's MMAs done
  uint64_t* acc_free = acc_full + 1;                                          // chunk drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acc_free + 1);
  if (warp == 0) qptc::tmem_alloc(tslot, 512);
  if (tid == 0) {
    for (int i = 0; i < F16_ST; ++i) {
      qptc::mbar_init(&a_full[i], NSW);
      qptc::mbar_init(&w_full[i], 1);
      qptc::mbar_init(&mma_done[i], 1);
    }
    qptc::mbar_init(acc_full, 1);
    qptc::mbar_init(acc_free, NSW);
  }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t t_main = tmem, t_corr = tmem + 256;

  // rows of a tile: nv = 4 -> 32 points x 4 vectors (row = vector * 32 + point), nv = 1 -> 128
  // points. Work items are (tile, column chunk) pairs; an item is nkc K stages.
  //  - MODE 1 (and small MODE 0 grids): items tile * ncc + chunk dealt round robin, so the CTAs
  //    holding the chunks of one tile run at the same time: the tile's costate rows are read
  //    from HBM once and its other reads hit L2.
  //  - MODE 0 with at least one tile per CTA: tiles dealt round robin, each CTA runs all
  //    chunks of its tile in turn (the row's tables are built once per tile).
  const int ppt = TM / a.nv;
  const int64_t ntiles = (a.npts + ppt - 1) / ppt;
  const bool tmaj = MODE == 0 && ntiles >= gridDim.x;
  const int64_t nitems = ntiles * ncc;
  const int my_items = tmaj ? (blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0) * ncc
                            : (blockIdx.x < nitems ? (int)((nitems - 1 - blockIdx.x) / gridDim.x) + 1 : 0);
  const int total = my_items * nkc;   // iterations of this CTA
  // (tile, column chunk) of item ki of this CTA
  auto item_tile = [&](int ki) -> int64_t {
    return tmaj ? blockIdx.x + (int64_t)(ki / ncc) * gridDim.x : (blockIdx.x + (int64_t)ki * gridDim.x) / ncc;
  };
  auto item_chunk = [&](int ki) -> int {
    return tmaj ? ki % ncc : (int)((blockIdx.x + (int64_t)ki * gridDim.x) % ncc);
  };
  bool ok = true;

  if (warp == NSW) {
    // ---- producer thread: the B block of iteration j once the MMAs of j - ST are done
    if (lane == 0) {
      int ji = 0, jk = 0;   // (item of this CTA, K stage) of iteration j
      int nj = 0;           // copies issued
      for (int j = 0; j < total && ok; ++j) {
        if (j >= F16_ST) ok = qptc::mbar_wait(&mma_done[j % F16_ST], (uint32_t)((j - F16_ST) / F16_ST) & 1);
        if (!ok) break;
        const int cj = item_chunk(ji);
        row16_copy_b<MODE>(B16, dim, ncc, cj, jk, sm + (j % F16_ST) * F16_STAGE + 2 * F16_ABYTES, &w_full[j % F16_ST]);
        nj = j + 1;
        if (++jk == nkc) { jk = 0; ++ji; }
      }
      if (!ok) {
        atomicExch(a.status, 6);
        // let this CTA's bulk copies land before exiting (the last ST issued at most)
        for (int j = nj - F16_ST < 0 ? 0 : nj - F16_ST; j < nj; ++j)
          qptc::mbar_wait(&w_full[j % F16_ST], (uint32_t)(j / F16_ST) & 1);
      }
    }
  } else if (warp == NSW + 1) {
    // ---- MMA thread: a stage's MMAs as soon as its operands are in shared memory
    if (lane == 0) {
      const uint32_t id = qptc::idesc(0, TM, 256);
      int last_commit = -1;
      int kc = 0, chunk = 0;
      for (int it = 0; it < total && ok; ++it) {
        const uint32_t st = (uint32_t)(it % F16_ST), ph = (uint32_t)(it / F16_ST) & 1;
        if (kc == 0 && chunk > 0) ok = qptc::mbar_wait(acc_free, (uint32_t)(chunk - 1) & 1);
        if (ok) ok = qptc::mbar_wait(&a_full[st], ph);
        if (ok) ok = qptc::mbar_wait(&w_full[st], ph);
        if (!ok) break;
        qptc::fence_after();
        const uint32_t sa = qptc::smem_u32(sm + st * F16_STAGE), sw = sa + 2 * F16_ABYTES;
#pragma unroll
        for (int ks = 0; ks < HKC / 16; ++ks) {
          const uint64_t ah = qptc::desc_kmajor(sa + ks * 256, 128, (HKC / 8) * 128);
          const uint64_t al = qptc::desc_kmajor(sa + F16_ABYTES + ks * 256, 128, (HKC / 8) * 128);
          const uint64_t wh = qptc::desc_kmajor(sw + ks * 256, 128, (HKC / 8) * 128);
          const uint64_t wl = qptc::desc_kmajor(sw + F16_WBYTES + ks * 256, 128, (HKC / 8) * 128);
          const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
          qptc::mma_f16(t_main, ah, wh, id, acc);
          qptc::mma_f16(t_corr, ah, wl, id, acc);
          qptc::mma_f16(t_corr, al, wh, id, 1u);
        }
        qptc::commit(&mma_done[st]);
        if (kc == nkc - 1) qptc::commit(acc_full);
        last_commit = it;
        if (++kc == nkc) { kc = 0; ++chunk; }
      }
      if (!ok) {
        atomicExch(a.status, 6);
        // let this CTA's tensor-core operations finish before tensor memory is freed
        if (last_commit >= 0)
          qptc::mbar_wait(&mma_done[last_commit % F16_ST], (uint32_t)(last_commit / F16_ST) & 1);
      }
    }
  } else {
    // ---- stager warps: tile row r (tensor-memory lane), half h of every K stage
    const int r = tid & (TM - 1), h = tid >> 7;
    const int s = a.nv == 4 ? r >> 5 : 0;
    const int prow = a.nv == 4 ? lane : r;
    const float sL = MODE == 1 ? pow2_scale(__int_as_float(__ldg(scal + 1))) : 1.f;
    float Lo[MODE == 0 ? 16 : 1], Lod[MODE == 0 ? 16 : 1];
    float hc[QP_MAXQ - 5], hsn[QP_MAXQ - 5], hj[QP_MAXQ - 5];
    // MODE 1 loads: instruction i of warp w reads tile rows lr(i) = 4 (4 w + i) + lane / 8, four
    // floats each at K offset 4 (lane % 8): 4 rows x 128 contiguous bytes per instruction.
    // Costate chunks of the next two iterations (even / odd iteration; two named arrays with
    // constant indices stay in registers).
    float4 pf0[MODE == 1 ? 4 : 1], pf1[MODE == 1 ? 4 : 1];
    auto lrow = [&](int i) { return 4 * (4 * warp + i) + (lane >> 3); };
    // costate chunk of tile row lr, iteration (item ki of this CTA, K stage kcj) (clamped for a
    // ragged tile)
    auto lam_src = [&](int ki, int kcj, int lr) -> const float4* {
      const int64_t tile = item_tile(ki);
      const int ls = a.nv == 4 ? lr >> 5 : 0;
      int64_t pj = tile * ppt + (a.nv == 4 ? (lr & 31) : lr);
      if (pj >= a.npts) pj = a.npts - 1;
      return reinterpret_cast<const float4*>(a.lam + ((a.pt_base + pj) * 4 + ls) * (int64_t)ktot + kcj * HKC +
                                             4 * (lane & 7));
    };
    // prefetch cursor (item, K stage) two iterations ahead of the current one
    int pki = 0, pkc = 0;
    auto adv = [&](int& ki, int& kk) {
      if (++kk == nkc) { kk = 0; ++ki; }
    };
    if (MODE == 1) {
      if (total > 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) pf0[i] = __ldg(lam_src(pki, pkc, lrow(i)));
        adv(pki, pkc);
      }
      if (total > 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) pf1[i] = __ldg(lam_src(pki, pkc, lrow(i)));
        adv(pki, pkc);
      }
    }
    float rs = sL, unsc = 1.f;
    float bmax = 0.f;   // MODE 0: largest row bound of this thread's active rows
    bool active = false;
    int64_t row = 0;
    int ki = 0, c = 0, kc = 0;
    int64_t cur_tile = -1;
    for (int it = 0; it < total && ok; ++it) {
      const uint32_t st = (uint32_t)(it % F16_ST);
      if (kc == 0) {
        // a new item: its column chunk; on a new tile its row and (MODE 0) the tables of the
        // row's product state and its scale
        const int64_t tile = item_tile(ki);
        c = item_chunk(ki);
        const int64_t p = tile * ppt + prow;
        active = p < a.npts;
        const int64_t pc = active ? p : a.npts - 1;
        row = (a.pt_base + pc) * 4 + s;
        if (MODE == 0 && tile != cur_tile) {
          cur_tile = tile;
          const float2* csp = a.cs ? a.cs + (a.pt_base + pc) * n : nullptr;
          const float4* tj = reinterpret_cast<const float4*>(a.thetaJ) + (a.pt_base + pc) * n;
          float jsum = 0.f;
#pragma unroll
          for (int t = 0; t < 16; ++t) { Lo[t] = 1.f; Lod[t] = 0.f; }
          for (int b = 0; b < 5; ++b) {
            const float4 tq = tj[n - 1 - b];
            float sn, cs;
            if (csp) {
              const float2 q2 = csp[n - 1 - b];
              cs = q2.x; sn = q2.y;
            } else {
              sincosf(0.5f * tq.x, &sn, &cs);
            }
            const float J = s == 1 ? tq.y : (s == 2 ? tq.z : tq.w);
            jsum += fabsf(J);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const bool bit = ((16 * h + t) >> b) & 1;
              const float f = bit ? sn : cs, d = bit ? 0.5f * cs : -0.5f * sn;
              Lod[t] = Lod[t] * f + Lo[t] * d * J;
              Lo[t] *= f;
            }
          }
#pragma unroll
          for (int q = 0; q < QP_MAXQ - 5; ++q) {
            hc[q] = 1.f; hsn[q] = 0.f; hj[q] = 0.f;
            if (q < high) {
              const float4 tq = tj[q];
              if (csp) {
                const float2 q2 = csp[q];
                hc[q] = q2.x; hsn[q] = q2.y;
              } else {
                sincosf(0.5f * tq.x, &hsn[q], &hc[q]);
              }
              hj[q] = s == 1 ? tq.y : (s == 2 ? tq.z : tq.w);
              jsum += fabsf(hj[q]);
            }
          }
          const float bound = s == 0 ? 1.f : 0.5f * jsum;
          rs = pow2_scale(bound);
          if (active) bmax = fmaxf(bmax, bound);
        }
        unsc = 1.f / (rs * W16_SCALE);
      }
      float v[HKC / 2];
      if (MODE == 0) {
        // high-bit factor of this K stage (qubit q <-> bit high-1-q of kc) and its derivative,
        // with the row's scale folded in
        float H = rs, Hd = 0.f;
#pragma unroll
        for (int q = 0; q < QP_MAXQ - 5; ++q) {
          if (q < high) {
            const bool bit = (kc >> (high - 1 - q)) & 1;
            const float f = bit ? hsn[q] : hc[q], d = bit ? 0.5f * hc[q] : -0.5f * hsn[q];
            Hd = Hd * f + H * d * hj[q];
            H *= f;
          }
        }
#pragma unroll
        for (int t = 0; t < HKC / 2; ++t) v[t] = s == 0 ? H * Lo[t] : Hd * Lo[t] + H * Lod[t];
      } else {
        const bool odd = it & 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 x = odd ? pf1[i] : pf0[i];
          v[4 * i] = x.x * rs; v[4 * i + 1] = x.y * rs; v[4 * i + 2] = x.z * rs; v[4 * i + 3] = x.w * rs;
        }
        if (it + 2 < total) {   // the slot is free again: the chunk two iterations ahead
          if (odd) {
#pragma unroll
            for (int i = 0; i < 4; ++i) pf1[i] = __ldg(lam_src(pki, pkc, lrow(i)));
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) pf0[i] = __ldg(lam_src(pki, pkc, lrow(i)));
          }
          adv(pki, pkc);
        }
      }
      // the stage's A region is free once the MMAs of iteration it - ST have finished
      bool good = true;
      if (it >= F16_ST) good = qptc::mbar_wait(&mma_done[st], (uint32_t)((it - F16_ST) / F16_ST) & 1);
      ok = __all_sync(0xffffffffu, good);
      if (!ok) break;
      unsigned char* sA = sm + st * F16_STAGE;
      if (MODE == 0) {
#pragma unroll
        for (int g8 = 0; g8 < HKC / 16; ++g8) {
          uint4 h8, l8;
          pack_h8(v + 8 * g8, 1.f, h8, l8);
          const uint32_t off = core_off_h(r, h * (HKC / 2) + g8 * 8);
          *reinterpret_cast<uint4*>(sA + off) = h8;
          *reinterpret_cast<uint4*>(sA + F16_ABYTES + off) = l8;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          uint4 h8, l8;   // only the first half of the eight-value pack is used
          float w8[8] = {v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3], 0.f, 0.f, 0.f, 0.f};
          pack_h8(w8, 1.f, h8, l8);
          const uint32_t off = core_off_h(lrow(i), 4 * (lane & 7));
          *reinterpret_cast<uint2*>(sA + off) = make_uint2(h8.x, h8.y);
          *reinterpret_cast<uint2*>(sA + F16_ABYTES + off) = make_uint2(l8.x, l8.y);
        }
      }
      qptc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) qptc::mbar_arrive(&a_full[st]);
      if (kc == nkc - 1) {
        // epilogue of this column chunk: both accumulators back, summed, unscaled (this
        // thread: its row, column half h)
        ok = __all_sync(0xffffffffu, qptc::mbar_wait(acc_full, (uint32_t)ki & 1));
        if (!ok) break;
        qptc::fence_after();
        float* orow = (MODE == 0 ? reinterpret_cast<float*>(a.phi) : a.mu) + row * (int64_t)ntot + c * 256 + h * 128;
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        for (int c0 = 0; c0 < 128; c0 += 32) {
          float vm[32], vc[32];
          qptc::tmem_ld32(t_main + lanes + h * 128 + c0, vm);
          qptc::tmem_ld32(t_corr + lanes + h * 128 + c0, vc);
          if (active) {
            float4* dst = reinterpret_cast<float4*>(orow + c0);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              dst[e] = make_float4((vm[4 * e] + vc[4 * e]) * unsc, (vm[4 * e + 1] + vc[4 * e + 1]) * unsc,
                                   (vm[4 * e + 2] + vc[4 * e + 2]) * unsc, (vm[4 * e + 3] + vc[4 * e + 3]) * unsc);
          }
        }
        qptc::fence_before();
        __syncwarp();
        if (lane == 0) qptc::mbar_arrive(acc_free);   // the accumulators are free for the next item
      }
      if (++kc == nkc) { kc = 0; ++ki; }
    }
    if (MODE == 0 && scal && h == 0) {   // one atomic per warp (same-address atomics serialise in L2)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
      if (lane == 0 && bmax > 0.f) atomicMax(scal, __float_as_int(bmax));
    }
    if (!ok && lane == 0) atomicExch(a.status, 6);
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------------- readout + head
struct ReadoutArgs {
  const float2* phi;
  const float* head;       // W[3][m], b[3]
  int32_t n, m, nv;
  int64_t npts, pt_base;
  float* out_f;            // [B][3]
  float* out_df;           // [B][3][3] or null
};

// Warp per point: z_i = sum_k |phi_k|^2 s_i(k), d z_i/dv_d = 2 sum_k Re(conj(phi_d,k) phi_k) s_i(k)
// (logical basis: the fused unitary already contains the CNOT rings), then the linear head.
__global__ void dense_readout_kernel(ReadoutArgs a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int n = a.n, dim = 1 << n, m = a.m;
  for (int64_t p = warp; p < a.npts; p += nw) {
    const float2* ph = a.phi + (a.pt_base + p) * 4 * dim;
    float z[QP_MAXQ], dz[3][QP_MAXQ];
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) { z[i] = 0.f; dz[0][i] = dz[1][i] = dz[2][i] = 0.f; }
#pragma unroll 4
    for (int k = lane; k < dim; k += 32) {
      const float2 f0 = ph[k];
      const float pr = f0.x * f0.x + f0.y * f0.y;
      float q[3] = {0.f, 0.f, 0.f};
      if (a.nv == 4) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float2 fd = ph[(1 + d) * dim + k];
          q[d] = 2.f * (fd.x * f0.x + fd.y * f0.y);
        }
      }
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i) {
        if (i < m) {
          const float sg = ((k >> (n - 1 - i)) & 1) ? -1.f : 1.f;
          z[i] += sg * pr;
#pragma unroll
          for (int d = 0; d < 3; ++d) dz[d][i] += sg * q[d];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) {
      if (i < m) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          z[i] += __shfl_xor_sync(0xffffffffu, z[i], o);
#pragma unroll
          for (int d = 0; d < 3; ++d) dz[d][i] += __shfl_xor_sync(0xffffffffu, dz[d][i], o);
        }
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float acc = a.head[3 * m + c], ad[3] = {0.f, 0.f, 0.f};
        for (int i = 0; i < m; ++i) {
          const float w = a.head[c * m + i];
          acc += w * z[i];
#pragma unroll
          for (int d = 0; d < 3; ++d) ad[d] += w * dz[d][i];
        }
        a.out_f[p * 3 + c] = acc;
        if (a.out_df && a.nv == 4) {
#pragma unroll
          for (int d = 0; d < 3; ++d) a.out_df[p * 9 + c * 3 + d] = ad[d];
        }
      }
    }
  }
}

}  // namespace qpd

namespace qpd {

// ------------------------------------------------------------------------- pointwise costates
// Warp per point: readout and head from Phi, loss terms and cotangents (shared with the SIMT
// path), head gradients, then the costates written over Phi in place:
//   lambda_0 = O phi_0 + sum_d O_d phi_d,  lambda_d = O_d phi_0,  O = sum_i zbar_i Z_i.
struct PointArgs {
  float2* phi;
  const float* head;
  int32_t n, m;
  const float* pts[3];
  int64_t npts[3], pt_base[3];
  QPProblemDev pb;
  const int32_t* counts;
  double* blk_loss;
  float* blk_grad;
  int32_t loss_stride, grad_stride, nE;
  int32_t* lmax;          // float bits of the largest |lambda| component (atomic maximum), or null
  // symmetry penalty (Eq. 18): cotangents added to the collocation points' fields (gsym) and
  // given for the rows of set 2 from nbc on (gext, the mirrored points); null without it
  const float* gsym;
  const float* gext;
  int64_t nbc;
};

// 8 warps per SM: a point's states (32 KiB at n = 10) are read twice, and the second read
// should hit L2; twice as many warps in flight measured 40% slower
constexpr int PT_POINT_THREADS = 256;
// NQ = n (9 or 10; the fused kernel covers 7 and 8). Lane l holds amplitudes k = l + 32 j: the
// sign of qubit i < n - 5 is bit n - 6 - i of j (a compile-time constant in the unrolled
// loops), that of qubit i >= n - 5 bit n - 1 - i of the lane. Both passes load PT_JB
// amplitudes of each vector before using them, so the loads of a batch are in flight together
// (the costate stores of pass 2 would otherwise order every load behind the previous store).
constexpr int PT_JB = 8;
template <int NQ>
__global__ void __launch_bounds__(PT_POINT_THREADS, 1) dense_point_kernel(PointArgs a) {
  static_assert(NQ >= 9 && NQ <= QP_MAXQ, "point kernel of the 9- and 10-qubit path");
  extern __shared__ __align__(16) unsigned char psh[];
  constexpr int n = NQ, dim = 1 << n, NJ = dim / 32, NH = n - 5;
  const int m = a.m;
  const int nt = a.pb.energy_nt;
  double* sloss = reinterpret_cast<double*>(psh);
  float* hacc = reinterpret_cast<float*>(psh + ((QP_NLP + nt) * 8 + 15) / 16 * 16);
  for (int i = threadIdx.x; i < QP_NLP + nt; i += blockDim.x) sloss[i] = 0.0;
  for (int i = threadIdx.x; i < 3 * m + 3; i += blockDim.x) hacc[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = a.npts[0] + a.npts[1] + a.npts[2];
  float lm = 0.f;   // largest |lambda| component this lane wrote
  for (int64_t gq = wg; gq < total; gq += nw) {
    int set = 0;
    int64_t li = gq;
    if (li >= a.npts[0]) { li -= a.npts[0]; set = 1; if (li >= a.npts[1]) { li -= a.npts[1]; set = 2; } }
    const bool v4 = set == 0;
    float2* ph = a.phi + (a.pt_base[set] + li) * 4 * dim;
    // ---- pass 1: |phi_0|^2 and 2 Re(phi_d^* phi_0) summed over this lane's amplitudes, with
    // the signs of the high qubits applied per j and those of the low qubits after the loop
    float tp = 0.f, tq[3] = {0.f, 0.f, 0.f}, hp[NH], hq[3][NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) { hp[i] = 0.f; hq[0][i] = hq[1][i] = hq[2][i] = 0.f; }
#pragma unroll
    for (int j0 = 0; j0 < NJ; j0 += PT_JB) {
      float2 f0[PT_JB], fd[3][PT_JB];
#pragma unroll
      for (int u = 0; u < PT_JB; ++u) {
        const int k = lane + 32 * (j0 + u);
        f0[u] = ph[k];
#pragma unroll
        for (int d = 0; d < 3; ++d) fd[d][u] = v4 ? ph[(1 + d) * dim + k] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < PT_JB; ++u) {
        const int j = j0 + u;
        const float pr = f0[u].x * f0[u].x + f0[u].y * f0[u].y;
        float q[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) q[d] = 2.f * (fd[d][u].x * f0[u].x + fd[d][u].y * f0[u].y);
        tp += pr;
#pragma unroll
        for (int d = 0; d < 3; ++d) tq[d] += q[d];
#pragma unroll
        for (int i = 0; i < NH; ++i) {
          const bool neg = (j >> (NH - 1 - i)) & 1;
          hp[i] += neg ? -pr : pr;
#pragma unroll
          for (int d = 0; d < 3; ++d) hq[d][i] += neg ? -q[d] : q[d];
        }
      }
    }
    float z[QP_MAXQ], dz[3][QP_MAXQ];
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) {
      float sv = 0.f, sd[3] = {0.f, 0.f, 0.f};
      if (i < NH) {
        sv = hp[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) sd[d] = hq[d][i];
      } else if (i < n) {
        const bool neg = (lane >> (n - 1 - i)) & 1;
        sv = neg ? -tp : tp;
#pragma unroll
        for (int d = 0; d < 3; ++d) sd[d] = neg ? -tq[d] : tq[d];
      }
      z[i] = i < m ? sv : 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) dz[d][i] = i < m ? sd[d] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i)
      if (i < m) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          z[i] += __shfl_xor_sync(0xffffffffu, z[i], o);
#pragma unroll
          for (int d = 0; d < 3; ++d) dz[d][i] += __shfl_xor_sync(0xffffffffu, dz[d][i], o);
        }
      }
    float f[3], D[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float acc = a.head[3 * m + c], ad[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i)
        if (i < m) {
          const float w = a.head[c * m + i];
          acc += w * z[i];
#pragma unroll
          for (int d = 0; d < 3; ++d) ad[d] += w * dz[d][i];
        }
      f[c] = acc;
#pragma unroll
      for (int d = 0; d < 3; ++d) D[c][d] = ad[d];
    }
    const float* xp = a.pts[set] + li * 3;
    float g[3], gD[3][3];
    const bool given = set == 2 && a.gext != nullptr && li >= a.nbc;
    qpk::point_loss(a.pb, set, li, set == 2 && a.gext != nullptr ? a.nbc : a.npts[set], a.counts, xp[0], xp[1], f, D,
                    !given, lane == 0, sloss, g, gD);
    if (given) {
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] = __ldg(a.gext + (li - a.nbc) * 3 + c);
    }
    if (set == 0 && a.gsym != nullptr) {
#pragma unroll
      for (int c = 0; c < 3; ++c) g[c] += __ldg(a.gsym + li * 3 + c);
    }
    float zb[QP_MAXQ], zbd[3][QP_MAXQ];
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) {
      zb[i] = 0.f;
      zbd[0][i] = zbd[1][i] = zbd[2][i] = 0.f;
      if (i < m) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float w = a.head[c * m + i];
          zb[i] += w * g[c];
#pragma unroll
          for (int d = 0; d < 3; ++d) zbd[d][i] += w * gD[c][d];
        }
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // constant indices keep z and dz in registers
#pragma unroll
        for (int i = 0; i < QP_MAXQ; ++i)
          if (i < m)
            atomicAdd(&hacc[c * m + i], g[c] * z[i] + gD[c][0] * dz[0][i] + gD[c][1] * dz[1][i] + gD[c][2] * dz[2][i]);
        atomicAdd(&hacc[3 * m + c], g[c]);
      }
    }
    // ---- pass 2: costates; O(k) = (low-qubit part of this lane) + (high-qubit part of j)
    // (zb and zbd are zero for the qubits that are not read out)
    float Ol = 0.f, Odl[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = NH; i < n; ++i) {
      const bool neg = (lane >> (n - 1 - i)) & 1;
      Ol += neg ? -zb[i] : zb[i];
#pragma unroll
      for (int d = 0; d < 3; ++d) Odl[d] += neg ? -zbd[d][i] : zbd[d][i];
    }
#pragma unroll
    for (int j0 = 0; j0 < NJ; j0 += PT_JB) {
      float2 f0[PT_JB], fd[3][PT_JB];
#pragma unroll
      for (int u = 0; u < PT_JB; ++u) {
        const int k = lane + 32 * (j0 + u);
        f0[u] = ph[k];
#pragma unroll
        for (int d = 0; d < 3; ++d) fd[d][u] = v4 ? ph[(1 + d) * dim + k] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < PT_JB; ++u) {
        const int j = j0 + u, k = lane + 32 * j;
        float O = Ol, Od[3] = {Odl[0], Odl[1], Odl[2]};
#pragma unroll
        for (int i = 0; i < NH; ++i) {
          const bool neg = (j >> (NH - 1 - i)) & 1;
          O += neg ? -zb[i] : zb[i];
#pragma unroll
          for (int d = 0; d < 3; ++d) Od[d] += neg ? -zbd[d][i] : zbd[d][i];
        }
        float2 lam = make_float2(O * f0[u].x, O * f0[u].y);
        if (v4) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            lam.x += Od[d] * fd[d][u].x;
            lam.y += Od[d] * fd[d][u].y;
            const float2 ld = make_float2(Od[d] * f0[u].x, Od[d] * f0[u].y);
            ph[(1 + d) * dim + k] = ld;
            lm = fmaxf(lm, fmaxf(fabsf(ld.x), fabsf(ld.y)));
          }
        }
        ph[k] = lam;
        lm = fmaxf(lm, fmaxf(fabsf(lam.x), fabsf(lam.y)));
      }
    }
  }
  if (a.lmax) {   // one atomic per warp (same-address atomics serialise in L2)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lm = fmaxf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    if (lane == 0 && lm > 0.f) atomicMax(a.lmax, __float_as_int(lm));
  }
  __syncthreads();
  double* bl = a.blk_loss + (int64_t)blockIdx.x * a.loss_stride;
  for (int i = threadIdx.x; i < QP_NLP + nt; i += blockDim.x) bl[i] = sloss[i];
  float* bg = a.blk_grad + (int64_t)blockIdx.x * a.grad_stride;
  for (int i = threadIdx.x; i < a.nE; i += blockDim.x) bg[i] = 0.f;
  for (int i = threadIdx.x; i < 3 * m + 3; i += blockDim.x) bg[a.nE + i] = hacc[i];
}

// ------------------------------------------------------------------------- B-independent sweep
// G[k][j] = sum_chunks (part[.][k][2j] - i part[.][k][2j+1]) (FP64 over chunks);
// Y = U' G with U' the fused unitary including the embedding phase: Y = sum phi lambda^dag at
// the end of the circuit.
struct SweepArgs {
  const float* part;
  int32_t nchunks, n, L, ansatz;
  const double2* U;     // [dim][dim]
  float2* G;            // [dim][dim] scratch
  float2* Y;            // [dim][dim]
  const float* params;
  int64_t circ_off;
  float* eout;          // blk_grad block 0: E[(l n + q) * 3 + P], then the CRZ sums [L][ncz]
  const double2* gates; // [L][n][4] rotation gates from the build (cluster sweep)
  const float2* crz;    // CRZ mesh ansatze: [L][2^n] diagonal (cos, sin) of each layer's mesh
};

// CRZ mesh gradient sums of one diagonal element w = Im Y[k][k] (basis index k): Z_t += z_t(k) w
// for every qubit t and Z_ct += z_c(k) z_t(k) w for every pair c < t (z_q(k) = 1 - 2 b_q(k)),
// into zs[ncz] by shared-memory atomics.
__device__ __forceinline__ void crz_sums_add(float* zs, int n, int k, float w) {
  for (int t = 0; t < n; ++t) {
    const float zt = ((k >> (n - 1 - t)) & 1) ? -w : w;
    atomicAdd(&zs[t], zt);
    for (int c = 0; c < t; ++c)
      atomicAdd(&zs[n + qp_pair_index(n, c, t)], ((k >> (n - 1 - c)) & 1) ? -zt : zt);
  }
}

// Compensated FP32 accumulation (Neumaier): s + c carries the sum to about twice FP32
// precision without the FP64 pipe (conversions and FP64 adds are slow on this part).
using qpk::CSum;   // compensated FP32 sum (qp_aux.cuh)

// G[k][j] = conj(sum over partial slots of part[slot][k][2j + re|im]), in two passes: slot
// groups (grid.y) each give a compensated partial (re sum, re carry, im sum, im carry), then
// the groups are combined. Eight independent loads in flight per thread.
__global__ void dense_gsum_kernel(SweepArgs a, int32_t groups, float4* gpart) {
  const int dim = 1 << a.n;
  const int64_t tot = (int64_t)dim * dim;
  const int64_t cstride = (int64_t)dim * 2 * dim;  // floats between consecutive slots
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= tot) return;
  const int g = blockIdx.y;
  const int c0 = (int)((int64_t)g * a.nchunks / groups), c1 = (int)((int64_t)(g + 1) * a.nchunks / groups);
  const int64_t k = e / dim, j = e % dim;
  const float* r = a.part + k * (2 * dim) + 2 * j;
  CSum re[2], im[2];
  int c = c0;
  for (; c + 8 <= c1; c += 8) {
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(reinterpret_cast<const float2*>(r + (int64_t)(c + u) * cstride));
#pragma unroll
    for (int u = 0; u < 8; ++u) { re[u & 1].add(v[u].x); im[u & 1].add(-v[u].y); }
  }
  for (; c < c1; ++c) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(r + (int64_t)c * cstride));
    re[0].add(v.x);
    im[0].add(-v.y);
  }
  re[0].add(re[1]);
  im[0].add(im[1]);
  gpart[(int64_t)g * tot + e] = make_float4(re[0].s, re[0].c, im[0].s, im[0].c);
}

__global__ void dense_gsum_fin_kernel(SweepArgs a, int32_t groups, const float4* gpart) {
  const int dim = 1 << a.n;
  const int64_t tot = (int64_t)dim * dim;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    CSum re, im;
    for (int g = 0; g < groups; ++g) {
      const float4 p = gpart[(int64_t)g * tot + e];
      CSum pr, pi;
      pr.s = p.x; pr.c = p.y; pi.s = p.z; pi.c = p.w;
      re.add(pr);
      im.add(pi);
    }
    a.G[e] = make_float2(re.value(), im.value());
  }
}

// Y[j][jj] = sum_k U'[j][k] G[k][jj], 16 x 16 output tiles, FP32 accumulation.
__global__ void dense_y_kernel(SweepArgs a) {
  const int dim = 1 << a.n;
  __shared__ float2 tu[16][17], tg[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int j = blockIdx.y * 16 + ty, jj = blockIdx.x * 16 + tx;
  float2 acc = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < dim; k0 += 16) {
    const double2 u = a.U[(int64_t)(blockIdx.y * 16 + ty) * dim + k0 + tx];
    tu[ty][tx] = make_float2((float)u.x, (float)u.y);
    tg[ty][tx] = a.G[(int64_t)(k0 + ty) * dim + blockIdx.x * 16 + tx];
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float2 x = tu[ty][kk], y = tg[kk][tx];
      acc.x += x.x * y.x - x.y * y.y;
      acc.y += x.x * y.y + x.y * y.x;
    }
    __syncthreads();
  }
  if (j < dim && jj < dim) a.Y[(int64_t)j * dim + jj] = acc;
}

// Undo ring l (Y2[a][b] = Y[c(a)][c(b)], i.e. C^dag Y C) and accumulate, at that point,
// E_P(l, q) = Im Tr(P_q Y2) for all q: Tr(X_q Y) = sum_a Y[a^q][a],
// Tr(Y_q Y) = sum_a (bit_q(a) ? i : -i) Y[a^q][a], Tr(Z_q Y) = sum_a (bit_q(a) ? -1 : 1) Y[a][a].
// For the CRZ mesh ansatze the layer ends with a diagonal D instead: Y2 = D^dag Y D, i.e.
// Y2[a][b] = conj(d_a) Y[a][b] d_b, and the mesh's gradient sums come from the diagonal.
__global__ void dense_sweep_ring_kernel(SweepArgs a, int l, const float2* Yin, float2* Yout) {
  const int n = a.n, dim = 1 << n;
  const int64_t tot = (int64_t)dim * dim;
  const bool crz = qp_has_crz(a.ansatz);
  const int ncz = qp_crz_sums(a.ansatz, n);
  __shared__ float es[QP_MAXQ * 3 + QP_MAXQ + QP_MAXQ * (QP_MAXQ - 1) / 2];
  float* zs = es + n * 3;
  for (int i = threadIdx.x; i < n * 3 + ncz; i += blockDim.x) es[i] = 0.f;
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int ra = (int)(e / dim), cb = (int)(e % dim);
    float2 v;
    if (crz) {
      const float2 y = Yin[e];
      const float2 da = a.crz[(int64_t)l * dim + ra], db = a.crz[(int64_t)l * dim + cb];
      const float2 t = make_float2(da.x * y.x + da.y * y.y, da.x * y.y - da.y * y.x);  // conj(da) y
      v = make_float2(t.x * db.x - t.y * db.y, t.x * db.y + t.y * db.x);
      if (ra == cb) crz_sums_add(zs, n, cb, y.y);
    } else {
      v = Yin[(int64_t)ring_map(n, a.ansatz, l, ra) * dim + ring_map(n, a.ansatz, l, cb)];
    }
    Yout[e] = v;
    const int x = ra ^ cb;
    if (x == 0) {
      for (int q = 0; q < n; ++q) atomicAdd(&es[q * 3 + 2], ((cb >> (n - 1 - q)) & 1) ? -v.y : v.y);
    } else if ((x & (x - 1)) == 0) {
      const int q = n - 1 - (31 - __clz(x));
      // element Y[a^q][a] with a = cb
      atomicAdd(&es[q * 3 + 0], v.y);
      atomicAdd(&es[q * 3 + 1], ((cb >> (n - 1 - q)) & 1) ? v.x : -v.x);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * 3; i += blockDim.x) atomicAdd(&a.eout[l * n * 3 + i], es[i]);
  for (int i = threadIdx.x; i < ncz; i += blockDim.x) atomicAdd(&a.eout[3 * n * a.L + l * ncz + i], zs[i]);
}

// Y <- R^dag Y (rows, TCOL-column tiles per block) for the rotations of layer l.
template <int TCOL>
__global__ void dense_sweep_left_kernel(SweepArgs a, int l, float2* Y) {
  extern __shared__ __align__(16) float2 tile[];  // [dim][TCOL]
  __shared__ double2 g[QP_MAXQ][4];
  const int n = a.n, dim = 1 << n;
  const int c0 = blockIdx.x * TCOL;
  if (threadIdx.x < n) gate_fp64(a.params, a.circ_off, a.ansatz, n, l, threadIdx.x, g[threadIdx.x]);
  for (int e = threadIdx.x; e < dim * TCOL; e += blockDim.x) tile[e] = Y[(int64_t)(e / TCOL) * dim + c0 + e % TCOL];
  __syncthreads();
  for (int q = 0; q < n; ++q) {
    const int bit = 1 << (n - 1 - q);
    const float2 u00 = make_float2((float)g[q][0].x, (float)g[q][0].y), u01 = make_float2((float)g[q][1].x, (float)g[q][1].y);
    const float2 u10 = make_float2((float)g[q][2].x, (float)g[q][2].y), u11 = make_float2((float)g[q][3].x, (float)g[q][3].y);
    for (int e = threadIdx.x; e < dim / 2 * TCOL; e += blockDim.x) {
      const int ri = e / TCOL, c = e % TCOL;
      const int r0 = ((ri & ~(bit - 1)) << 1) | (ri & (bit - 1)), r1 = r0 | bit;
      const float2 x = tile[r0 * TCOL + c], y = tile[r1 * TCOL + c];
      tile[r0 * TCOL + c] = make_float2(u00.x * x.x + u00.y * x.y + u10.x * y.x + u10.y * y.y,
                                        u00.x * x.y - u00.y * x.x + u10.x * y.y - u10.y * y.x);
      tile[r1 * TCOL + c] = make_float2(u01.x * x.x + u01.y * x.y + u11.x * y.x + u11.y * y.y,
                                        u01.x * x.y - u01.y * x.x + u11.x * y.y - u11.y * y.x);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < dim * TCOL; e += blockDim.x) Y[(int64_t)(e / TCOL) * dim + c0 + e % TCOL] = tile[e];
}

// Y <- Y R (columns, TROW-row tiles per block) for the rotations of layer l.
template <int TROW>
__global__ void dense_sweep_right_kernel(SweepArgs a, int l, float2* Y) {
  extern __shared__ __align__(16) float2 tile[];  // [TROW][dim]
  __shared__ double2 g[QP_MAXQ][4];
  const int n = a.n, dim = 1 << n;
  const int r0b = blockIdx.x * TROW;
  if (threadIdx.x < n) gate_fp64(a.params, a.circ_off, a.ansatz, n, l, threadIdx.x, g[threadIdx.x]);
  for (int e = threadIdx.x; e < dim * TROW; e += blockDim.x) tile[e] = Y[(int64_t)r0b * dim + e];
  __syncthreads();
  for (int q = 0; q < n; ++q) {
    const int bit = 1 << (n - 1 - q);
    const float2 u00 = make_float2((float)g[q][0].x, (float)g[q][0].y), u01 = make_float2((float)g[q][1].x, (float)g[q][1].y);
    const float2 u10 = make_float2((float)g[q][2].x, (float)g[q][2].y), u11 = make_float2((float)g[q][3].x, (float)g[q][3].y);
    for (int e = threadIdx.x; e < dim / 2 * TROW; e += blockDim.x) {
      const int row = e / (dim / 2), ci = e % (dim / 2);
      const int c0 = ((ci & ~(bit - 1)) << 1) | (ci & (bit - 1)), c1 = c0 | bit;
      const float2 x = tile[row * dim + c0], y = tile[row * dim + c1];
      tile[row * dim + c0] = make_float2(x.x * u00.x - x.y * u00.y + y.x * u10.x - y.y * u10.y,
                                         x.x * u00.y + x.y * u00.x + y.x * u10.y + y.y * u10.x);
      tile[row * dim + c1] = make_float2(x.x * u01.x - x.y * u01.y + y.x * u11.x - y.y * u11.y,
                                         x.x * u01.y + x.y * u01.x + y.x * u11.y + y.y * u11.x);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < dim * TROW; e += blockDim.x) Y[(int64_t)r0b * dim + e] = tile[e];
}


// ---- whole sweep in one thread-block cluster (n <= 8: Y fits the cluster's shared memory)
// The S CTAs of the cluster hold Y (2^n x 2^n) in two layouts, w = 2^n / S indices each:
//   C (columns): CTA c holds Y[row][c w + j] for every row, at bufC[row][j],
//   R (rows):    CTA c holds Y[c w + i][col] for every column, at bufR[col][i],
// both stored [full index x][local index j] with j swizzled by x (j ^ (x mod w)), so that
// the row-wise gate passes, the column-wise gate passes and the transposing gathers between
// the layouts all read and write shared memory without bank conflicts. Per layer l (last to
// first): the CNOT ring is undone by gathering C from R across the cluster, E(l) is read off
// C, the rotations are undone on the rows in C (R^dag Y) and, after a gather back to R, on
// the columns (Y R). Two cluster barriers per layer; one launch for the whole sweep.
constexpr int SWC_THREADS = 512;
constexpr int SWC_UNROLL = 8;     // cluster loads in flight per thread
// cluster size: 2^n CTAs up to 8, or 16 where the GPU can co-schedule a 16-CTA cluster
__host__ __device__ inline int swc_size(int n, bool big) {
  const int cap = big ? 16 : 8;
  return (1 << n) < cap ? (1 << n) : cap;
}
__host__ __device__ inline int swc_smem(int n, int L, int S, int ncz) {
  const int dim = 1 << n, w = dim / S;
  return 2 * dim * w * 8 + L * n * 4 * 8 + 2 * dim * 4 + L * n * 3 * 4 + L * ncz * 4;
}
__device__ __forceinline__ int swz(int x, int j, int w) { return x * w + (j ^ (x & (w - 1))); }

// One pass of the gates of qubits q0 .. q0 + g - 1 (g <= 4) over the full index x of a
// [2^n][w] buffer: each thread carries the 2^g elements of one (x outside the group, j) in
// registers. y0 = u00 x0 + u10 x1, y1 = u01 x0 + u11 x1 with u conjugated when `dag`.
__device__ __forceinline__ void swc_gates(float2* buf, int n, int w, int q0, int g, const float2* gl, bool dag) {
  const int dim = 1 << n, plo = n - q0 - g, ng = 1 << g;
  const int ngrp = (dim >> g) * w;
  for (int t = threadIdx.x; t < ngrp; t += blockDim.x) {
    const int j = t % w, rest = t / w;
    const int xb = ((rest >> plo) << (plo + g)) | (rest & ((1 << plo) - 1));
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if (m < ng) v[m] = buf[swz(xb | (m << plo), j, w)];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (b < g) {
        // qubit q0 + g - 1 - b owns bit b of m
        const float2* u = gl + (q0 + g - 1 - b) * 4;
        const float sy = dag ? -1.f : 1.f;
        const float2 u00 = make_float2(u[0].x, sy * u[0].y), u01 = make_float2(u[1].x, sy * u[1].y);
        const float2 u10 = make_float2(u[2].x, sy * u[2].y), u11 = make_float2(u[3].x, sy * u[3].y);
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          if (m < ng && !((m >> b) & 1)) {
            const float2 x0 = v[m], x1 = v[m | (1 << b)];
            v[m] = make_float2(u00.x * x0.x - u00.y * x0.y + u10.x * x1.x - u10.y * x1.y,
                               u00.x * x0.y + u00.y * x0.x + u10.x * x1.y + u10.y * x1.x);
            v[m | (1 << b)] = make_float2(u01.x * x0.x - u01.y * x0.y + u11.x * x1.x - u11.y * x1.y,
                                          u01.x * x0.y + u01.y * x0.x + u11.x * x1.y + u11.y * x1.x);
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if (m < ng) buf[swz(xb | (m << plo), j, w)] = v[m];
  }
}

__global__ void __launch_bounds__(SWC_THREADS) dense_sweep_cluster_kernel(SweepArgs a) {
  extern __shared__ __align__(16) float2 swsm[];
  const int n = a.n, dim = 1 << n, L = a.L;
  const int S = (int)qptc::cluster_size(), w = dim / S, lw = n - (31 - __clz(S));
  const int c = (int)qptc::cluster_rank();
  const int wi = threadIdx.x >> 5, ln = threadIdx.x & 31;
  float2* bufR = swsm;                          // [dim][w]
  float2* bufC = bufR + dim * w;                // [dim][w]
  float2* gm = bufC + dim * w;                  // [L][n][4] rotation gates (FP32)
  int* cmap = reinterpret_cast<int*>(gm + L * n * 4);   // ring map of the current layer
  int* cinv = cmap + dim;                                // and its inverse
  float* es = reinterpret_cast<float*>(cinv + dim);      // [L][n][3] E partials, [L][ncz] CRZ sums
  const bool crz = qp_has_crz(a.ansatz);
  const int ncz = qp_crz_sums(a.ansatz, n);
  // the whole cluster is resident: a kernel launched as this one's programmatic dependent (the
  // premap backward of the loss call) may take the other SMs now
  qptc::pdl_launch_dependents();
  for (int i = threadIdx.x; i < L * n * 4; i += blockDim.x) {
    const double2 g = a.gates[i];
    gm[i] = make_float2((float)g.x, (float)g.y);
  }
  for (int i = threadIdx.x; i < L * n * 3 + L * ncz; i += blockDim.x) es[i] = 0.f;
  // this CTA's rows of Y (row-major in global memory) into layout R
  for (int e0 = threadIdx.x; e0 < w * dim; e0 += SWC_UNROLL * blockDim.x) {
    float2 v[SWC_UNROLL];
#pragma unroll
    for (int u = 0; u < SWC_UNROLL; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < w * dim) v[u] = a.Y[(int64_t)(c * w + e / dim) * dim + e % dim];
    }
#pragma unroll
    for (int u = 0; u < SWC_UNROLL; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < w * dim) bufR[swz(e % dim, e / dim, w)] = v[u];
    }
  }
  qptc::cluster_sync();
  for (int l = L - 1; l >= 0; --l) {
    for (int k = threadIdx.x; k < dim; k += blockDim.x) {
      const int ck = ring_map(n, a.ansatz, l, k);
      cmap[k] = ck;
      cinv[ck] = k;
    }
    __syncthreads();
    // (1) Y2[ra][cb] = Y[c(ra)][c(cb)] for this CTA's columns cb = c w + j, into layout C. The
    // lanes walk the source rows c(ra) = owner w + i of one source column c(cb): one
    // contiguous row of the owner's layout R per warp access.
    for (int e0 = threadIdx.x; e0 < dim * w; e0 += SWC_UNROLL * blockDim.x) {
      float2 v[SWC_UNROLL];
#pragma unroll
      for (int u = 0; u < SWC_UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < dim * w) {
          const int i = e & (w - 1), j = (e >> lw) & (w - 1), owner = e >> (2 * lw);
          v[u] = qptc::cluster_ld_f2(qptc::cluster_map(&bufR[swz(cmap[c * w + j], i, w)], (uint32_t)owner));
        }
      }
#pragma unroll
      for (int u = 0; u < SWC_UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < dim * w) {
          const int i = e & (w - 1), j = (e >> lw) & (w - 1), owner = e >> (2 * lw);
          float2 y = v[u];
          if (crz) {
            // CRZ mesh: Y2[ra][cb] = conj(d_ra) Y[ra][cb] d_cb (the maps are the identity)
            const float2 da = __ldg(&a.crz[l * dim + owner * w + i]), db = __ldg(&a.crz[l * dim + c * w + j]);
            const float2 t = make_float2(da.x * y.x + da.y * y.y, da.x * y.y - da.y * y.x);
            y = make_float2(t.x * db.x - t.y * db.y, t.x * db.y + t.y * db.x);
          }
          bufC[swz(cinv[owner * w + i], j, w)] = y;
        }
      }
    }
    __syncthreads();
    // E_P(l, q) = Im Tr(P_q Y2): warp b <= n takes the off-diagonal elements Y2[cb ^ 2^b][cb]
    // (X and Y terms of qubit n - 1 - b) or, b = n, the diagonal (Z terms), lanes = columns
    if (wi <= n) {
      const bool act = ln < w;
      const int cb = c * w + (act ? ln : 0);
      float* el = es + l * n * 3;
      if (wi == n) {
        const float vy = act ? bufC[swz(cb, ln, w)].y : 0.f;
        for (int q = 0; q < n; ++q) {
          float t = ((cb >> (n - 1 - q)) & 1) ? -vy : vy;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (ln == 0) el[q * 3 + 2] += t;
        }
        if (crz) {
          // CRZ mesh sums from the same diagonal: Z_t and Z_ct for c < t
          float* zl = es + L * n * 3 + l * ncz;
          for (int t = 0; t < n; ++t) {
            const float zt = ((cb >> (n - 1 - t)) & 1) ? -vy : vy;
            float r = zt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (ln == 0) zl[t] += r;
            for (int c2 = 0; c2 < t; ++c2) {
              float r2 = ((cb >> (n - 1 - c2)) & 1) ? -zt : zt;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
              if (ln == 0) zl[n + qp_pair_index(n, c2, t)] += r2;
            }
          }
        }
      } else {
        const int q = n - 1 - wi;
        const float2 v = act ? bufC[swz(cb ^ (1 << wi), ln, w)] : make_float2(0.f, 0.f);
        float tx = v.y, ty = ((cb >> wi) & 1) ? v.x : -v.x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          tx += __shfl_xor_sync(0xffffffffu, tx, o);
          ty += __shfl_xor_sync(0xffffffffu, ty, o);
        }
        if (ln == 0) { el[q * 3 + 0] += tx; el[q * 3 + 1] += ty; }
      }
    }
    if (l == 0) break;
    __syncthreads();
    // (2) rows: Y <- R_l^dag Y
    const float2* gl = gm + l * n * 4;
    for (int q0 = 0; q0 < n; q0 += 4) {
      swc_gates(bufC, n, w, q0, n - q0 < 4 ? n - q0 : 4, gl, true);
      __syncthreads();
    }
    qptc::cluster_sync();
    // (3) back to layout R: Y[c w + i][col] sits in CTA col / w at bufC[c w + i][col mod w];
    // the lanes walk col mod w (one contiguous row of the owner's layout C per warp access)
    for (int e0 = threadIdx.x; e0 < dim * w; e0 += SWC_UNROLL * blockDim.x) {
      float2 v[SWC_UNROLL];
#pragma unroll
      for (int u = 0; u < SWC_UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < dim * w) {
          const int j = e & (w - 1), i = (e >> lw) & (w - 1), owner = e >> (2 * lw);
          v[u] = qptc::cluster_ld_f2(qptc::cluster_map(&bufC[swz(c * w + i, j, w)], (uint32_t)owner));
        }
      }
#pragma unroll
      for (int u = 0; u < SWC_UNROLL; ++u) {
        const int e = e0 + u * blockDim.x;
        if (e < dim * w) {
          const int j = e & (w - 1), i = (e >> lw) & (w - 1), owner = e >> (2 * lw);
          bufR[swz(owner * w + j, i, w)] = v[u];
        }
      }
    }
    __syncthreads();
    // (4) columns: Y <- Y R_l
    for (int q0 = 0; q0 < n; q0 += 4) {
      swc_gates(bufR, n, w, q0, n - q0 < 4 ? n - q0 : 4, gl, false);
      __syncthreads();
    }
    qptc::cluster_sync();
  }
  // every peer is done reading this CTA's layout R before it exits
  qptc::cluster_sync();
  for (int i = threadIdx.x; i < L * n * 3 + L * ncz; i += blockDim.x) atomicAdd(&a.eout[i], es[i]);
}
}  // namespace qpd

namespace qpd {

// Per-point embedding gradients from mu_s = Re(U'^H lambda_s). For both embeddings the folded
// phase D satisfies D^H G_q D = Y_q (G = X for RX with D = (-i)^{popcount}, G = Y for RY with
// D = 1), so with the real product-state vectors R_s:
//   dL/dtheta_q = sum_s Im<lambda_s|G_q psi_s> = sum_s sum_a sigma_q(a) R_s[a ^ q] mu_s[a],
//   dL/dJ_qd    = Im<lambda_d|G_q psi_0>      = sum_a sigma_q(a) R_0[a ^ q] mu_d[a],
// sigma_q(a) = +1 where qubit q of a is 1, -1 where it is 0. R_s[a ^ q] comes from prefix and
// suffix products of the per-qubit factors carried with their x, y, t derivatives.
struct EmbedArgs {
  const float* thetaJ;
  const float* mu;          // [P][4][dim]
  float* dthetaJ;           // [P][n] float4
  int32_t n;
  int64_t npts[3], pt_base[3];
  const float2* cs;         // [P][n] (cos, sin) of theta / 2
};

struct Dual4 {
  float v, d0, d1, d2;
};
__device__ __forceinline__ Dual4 dmul4(const Dual4& a, const Dual4& b) {
  return {a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1, a.d2 * b.v + a.v * b.d2};
}

// Embedding gradients from mu (n >= 5), warp per point. With the flipped-factor identity (the
// derivative of a qubit's cos/sin(theta/2) factor is the other one, halved and signed),
//   dL/dtheta_q = sum_k sign_q(k) [F_q(k).v mu_0[k] + sum_d F_q(k).d_d mu_d[k]],
//   dL/dJ_{q,d} = sum_k sign_q(k) F_q(k).v mu_d[k],
// with F_q(k) the product state's dual (value; x, y, t tangents) with qubit q's factor flipped
// and sign_q(k) = +1 where qubit q is 1. Split k = (hi, lo), lo the five lowest index bits:
// the product state is Hi(hi) x Lo(lo) and a flip stays inside one factor, so every sum is a
// 2^(n-5) x 32 table contraction; lane = lo, one pass over the rows hi of mu:
//   low q:  sum_lo sign [LF_q.v (A0 + sum_d B_d) + sum_d LF_q.d_d A_d],  A_d[lo] = sum_hi Hi.v mu_d,
//           A0 = sum_hi Hi.v mu_0, B_d = sum_hi Hi.d_d mu_d;
//   high q: sum_hi sign [HF_q.v (sum_lo Lo.v mu_0 + Lo.d_d mu_d) + sum_d HF_q.d_d sum_lo Lo.v mu_d].
constexpr int EG_WARPS = 8;
__global__ void __launch_bounds__(EG_WARPS * 32) dense_embed_grad_kernel(EmbedArgs a) {
  constexpr int NHQ = QP_MAXQ - 5;                       // high qubits at most
  __shared__ float4 tabs[EG_WARPS][NHQ + 1][32];         // per warp: Hi, then HF_q, over hi
  const int n = a.n, dim = 1 << n, nh = n - 5, nhi = dim >> 5;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  float4 (*tb)[32] = tabs[wl];
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = a.npts[0] + a.npts[1] + a.npts[2];
  for (int64_t gq = wg; gq < total; gq += nw) {
    int set = 0;
    int64_t li = gq;
    if (li >= a.npts[0]) { li -= a.npts[0]; set = 1; if (li >= a.npts[1]) { li -= a.npts[1]; set = 2; } }
    const bool nv4 = set == 0;
    const int64_t gp = a.pt_base[set] + li;
    // lane q < n holds qubit q's (cos, sin) of theta/2 and its J
    float cq = 1.f, sq = 0.f;
    float4 jq = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < n) {
      const float2 c2 = __ldg(a.cs + gp * n + lane);
      cq = c2.x; sq = c2.y;
      jq = __ldg(reinterpret_cast<const float4*>(a.thetaJ) + gp * n + lane);
    }
    // factor and flipped factor of qubit q at bit value `bit`, as duals (all lanes shuffle)
    auto factors = [&](int q, bool bit, Dual4& F, Dual4& G) {
      const float c = __shfl_sync(0xffffffffu, cq, q), sn = __shfl_sync(0xffffffffu, sq, q);
      const float jx = __shfl_sync(0xffffffffu, jq.y, q), jy = __shfl_sync(0xffffffffu, jq.z, q),
                  jt = __shfl_sync(0xffffffffu, jq.w, q);
      const float f = bit ? sn : c, d = bit ? 0.5f * c : -0.5f * sn;
      const float g = bit ? c : sn, e = bit ? -0.5f * sn : 0.5f * c;
      F = {f, d * jx, d * jy, d * jt};
      G = {g, e * jx, e * jy, e * jt};
    };
    // low factors of this lane's lo (qubit n - 1 - b <-> bit b), prefix / suffix products
    Dual4 LF[5], Lo;
    {
      Dual4 F[5], G[5], pre[6], suf[6];
#pragma unroll
      for (int b = 0; b < 5; ++b) factors(n - 1 - b, (lane >> b) & 1, F[b], G[b]);
      pre[0] = {1.f, 0.f, 0.f, 0.f};
      suf[5] = {1.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int b = 0; b < 5; ++b) pre[b + 1] = dmul4(pre[b], F[b]);
#pragma unroll
      for (int b = 4; b >= 0; --b) suf[b] = dmul4(F[b], suf[b + 1]);
      Lo = pre[5];
#pragma unroll
      for (int b = 0; b < 5; ++b) LF[b] = dmul4(dmul4(pre[b], G[b]), suf[b + 1]);
    }
    // high tables for hi = lane (qubit q < nh <-> bit nh - 1 - q of hi)
    {
      Dual4 F[NHQ], G[NHQ], pre[NHQ + 1], suf[NHQ + 1];
#pragma unroll
      for (int q = 0; q < NHQ; ++q) {
        F[q] = {1.f, 0.f, 0.f, 0.f};
        G[q] = {1.f, 0.f, 0.f, 0.f};
        if (q < nh) factors(q, (lane >> (nh - 1 - q)) & 1, F[q], G[q]);
      }
      pre[0] = {1.f, 0.f, 0.f, 0.f};
      suf[NHQ] = {1.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < NHQ; ++q) pre[q + 1] = dmul4(pre[q], F[q]);
#pragma unroll
      for (int q = NHQ - 1; q >= 0; --q) suf[q] = dmul4(F[q], suf[q + 1]);
      __syncwarp();   // the previous point's tables are read
      if (lane < nhi) {
        tb[0][lane] = make_float4(pre[NHQ].v, pre[NHQ].d0, pre[NHQ].d1, pre[NHQ].d2);
#pragma unroll
        for (int q = 0; q < NHQ; ++q)
          if (q < nh) {
            const Dual4 h = dmul4(dmul4(pre[q], G[q]), suf[q + 1]);
            tb[1 + q][lane] = make_float4(h.v, h.d0, h.d1, h.d2);
          }
      }
      __syncwarp();
    }
    // one pass over the rows of mu
    const float* mu = a.mu + gp * 4 * dim;
    float A0 = 0.f, Ad[3] = {0.f, 0.f, 0.f}, Bd[3] = {0.f, 0.f, 0.f};
    float gh[NHQ], gJh[3][NHQ];
#pragma unroll
    for (int q = 0; q < NHQ; ++q) { gh[q] = 0.f; gJh[0][q] = gJh[1][q] = gJh[2][q] = 0.f; }
    for (int hi = 0; hi < nhi; ++hi) {
      const int k = hi * 32 + lane;
      const float m0 = mu[k];
      float md[3] = {0.f, 0.f, 0.f};
      if (nv4) { md[0] = mu[dim + k]; md[1] = mu[2 * dim + k]; md[2] = mu[3 * dim + k]; }
      const float4 H = tb[0][hi];
      A0 += H.x * m0;
      Ad[0] += H.x * md[0]; Ad[1] += H.x * md[1]; Ad[2] += H.x * md[2];
      Bd[0] += H.y * md[0]; Bd[1] += H.z * md[1]; Bd[2] += H.w * md[2];
      const float t0 = Lo.v * m0 + Lo.d0 * md[0] + Lo.d1 * md[1] + Lo.d2 * md[2];
      const float td0 = Lo.v * md[0], td1 = Lo.v * md[1], td2 = Lo.v * md[2];
#pragma unroll
      for (int q = 0; q < NHQ; ++q) {
        if (q < nh) {
          const float4 HF = tb[1 + q][hi];
          const float sg = ((hi >> (nh - 1 - q)) & 1) ? 1.f : -1.f;
          gh[q] += sg * (HF.x * t0 + HF.y * td0 + HF.z * td1 + HF.w * td2);
          gJh[0][q] += sg * HF.x * td0;
          gJh[1][q] += sg * HF.x * td1;
          gJh[2][q] += sg * HF.x * td2;
        }
      }
    }
    // this lane's contributions: low qubits from its lo, high qubits from its pass
    float gth[QP_MAXQ], gJ[3][QP_MAXQ];
#pragma unroll
    for (int q = 0; q < QP_MAXQ; ++q) { gth[q] = 0.f; gJ[0][q] = gJ[1][q] = gJ[2][q] = 0.f; }
#pragma unroll
    for (int q = 0; q < NHQ; ++q) {
      if (q < nh) { gth[q] = gh[q]; gJ[0][q] = gJh[0][q]; gJ[1][q] = gJh[1][q]; gJ[2][q] = gJh[2][q]; }
    }
    const float AB = A0 + Bd[0] + Bd[1] + Bd[2];
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const float sg = ((lane >> b) & 1) ? 1.f : -1.f;
      const float gl = sg * (LF[b].v * AB + LF[b].d0 * Ad[0] + LF[b].d1 * Ad[1] + LF[b].d2 * Ad[2]);
#pragma unroll
      for (int q = 0; q < QP_MAXQ; ++q) {
        if (q == n - 1 - b) {
          gth[q] = gl;
          gJ[0][q] = sg * LF[b].v * Ad[0];
          gJ[1][q] = sg * LF[b].v * Ad[1];
          gJ[2][q] = sg * LF[b].v * Ad[2];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < QP_MAXQ; ++q) {
      if (q < n) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          gth[q] += __shfl_xor_sync(0xffffffffu, gth[q], o);
          gJ[0][q] += __shfl_xor_sync(0xffffffffu, gJ[0][q], o);
          gJ[1][q] += __shfl_xor_sync(0xffffffffu, gJ[1][q], o);
          gJ[2][q] += __shfl_xor_sync(0xffffffffu, gJ[2][q], o);
        }
        if (lane == 0)
          reinterpret_cast<float4*>(a.dthetaJ)[gp * n + q] = make_float4(gth[q], gJ[0][q], gJ[1][q], gJ[2][q]);
      }
    }
  }
}

}  // namespace qpd
