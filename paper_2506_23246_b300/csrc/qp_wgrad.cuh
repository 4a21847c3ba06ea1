// qp_wgrad.cuh -- weight-gradient contraction G = sum over (point, vector) rows of
// R Lambda^H on the tensor cores (3xTF32), FP32 partials per row chunk.
#pragma once
#include "qp_dense.cuh"

namespace qpd {

// ------------------------------------------------------------------------- weight-gradient GEMM
// G_part[chunk][k][o] = sum over the chunk's (point, vector) rows of R_s[k] * Lambda_s[o]:
// M = 128 basis indices k, N = 256 costate components o = (amp, re|im), K = (point, vector)
// rows, 32 per K-chunk. K-chunks never straddle point sets: a collocation chunk holds 8 points
// x 4 vectors (rows consecutive in the costate buffer), an IC/BC chunk 32 points x 1 vector.
// R is regenerated from the angles, one product-rule pass per point giving all four vectors.
struct WgArgs {
  const float* thetaJ;
  const float2* lam;          // [P][4][dim]
  float* part;                // [nchunks][dim][2 dim]
  int32_t n;
  int64_t npts[3], pt_base[3];
  int64_t kc_end[3];          // cumulative K-chunk counts per set
  int32_t nchunks;            // point-range chunks (grid.y)
  int32_t* status;
};

__host__ __device__ inline int wg_smem_bytes() { return 2 * (2 * TM * KC * 4 + 2 * 256 * KC * 4) + 128 + 32 * QP_MAXQ * 32; }

// Global loads of one K-chunk, issued one iteration ahead (software pipeline): the costate
// values this thread stages (component o = nt * 256 + tid of the chunk's 32 rows) and the raw
// angle entries (theta, J) of up to 2 (point, qubit) pairs of the chunk.
constexpr int WG_THREADS = 256;
struct WgPrefetch {
  float lam[KC];
  float4 tj[2];
};

__device__ __forceinline__ void wg_chunk_geom(const WgArgs& a, int64_t kc, int& set, int64_t& p0, int& ppc) {
  set = kc < a.kc_end[0] ? 0 : (kc < a.kc_end[1] ? 1 : 2);
  const int64_t ck = kc - (set == 0 ? 0 : a.kc_end[set - 1]);
  ppc = set == 0 ? 8 : 32;
  p0 = ck * ppc;
}

__device__ __forceinline__ void wg_prefetch(const WgArgs& a, int64_t kc, int tid, int o, WgPrefetch& f) {
  const int n = a.n, dim = 1 << n;
  int set, ppc;
  int64_t p0;
  wg_chunk_geom(a, kc, set, p0, ppc);
  const int64_t np = a.npts[set];
  const float* lamf = reinterpret_cast<const float*>(a.lam);
  const int64_t row0 = (a.pt_base[set] + p0) * 4;
  const int rstep = set == 0 ? 1 : 4;
  const int nvalid = set == 0 ? (int)((np - p0) * 4 < KC ? (np - p0) * 4 : KC) : (int)(np - p0 < KC ? np - p0 : KC);
#pragma unroll
  for (int t = 0; t < KC; ++t)
    f.lam[t] = t < nvalid ? __ldg(lamf + (row0 + (int64_t)t * rstep) * (2 * dim) + o) : 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int e = tid + j * WG_THREADS;
    const int pl = e / n, q = e % n;
    f.tj[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < ppc * n && p0 + pl < np)
      f.tj[j] = __ldg(reinterpret_cast<const float4*>(a.thetaJ) + (a.pt_base[set] + p0 + pl) * n + q);
  }
}

__global__ void __launch_bounds__(WG_THREADS, 1) dense_wgrad_gemm_kernel(WgArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int n = a.n, dim = 1 << n;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = blockIdx.x % (dim / TM), nt = blockIdx.x / (dim / TM);
  const int nch = 256;
  const int abytes = TM * KC * 4, bbytes = nch * KC * 4;
  const int stage_bytes = 2 * abytes + 2 * bbytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);  // mma_done[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage_bytes + 64);
  float4* fac = reinterpret_cast<float4*>(sm + 2 * stage_bytes + 128);  // [32 pts][n][2]
  if (warp == 0) qptc::tmem_alloc(tslot, 256);
  if (tid == 0) { qptc::mbar_init(&bars[0], 1); qptc::mbar_init(&bars[1], 1); }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = qptc::idesc(2, TM, nch);
  const int64_t nkc_total = a.kc_end[2];
  const int64_t per = (nkc_total + a.nchunks - 1) / a.nchunks;
  const int64_t kc0 = blockIdx.y * per;
  const int64_t kc1 = kc0 + per < nkc_total ? kc0 + per : nkc_total;
  const int arow = tid & (TM - 1), ahalf = tid >> 7;  // A row (basis index) and half of the chunk
  const int krow = mt * TM + arow;
  const int o = nt * nch + tid;                      // costate component staged by this thread
  bool ok = true;
  uint32_t it = 0;
  WgPrefetch pf;
  if (kc0 < kc1) wg_prefetch(a, kc0, tid, o, pf);
  for (int64_t kc = kc0; kc < kc1 && ok; ++kc, ++it) {
    const uint32_t st = it & 1;
    unsigned char* sA = sm + st * stage_bytes;
    unsigned char* sB = sA + 2 * abytes;
    int set, ppc;
    int64_t p0;
    wg_chunk_geom(a, kc, set, p0, ppc);
    bool w_ok = true;
    if (it >= 2) w_ok = qptc::mbar_wait(&bars[st], ((it - 2) >> 1) & 1);
    ok = __syncthreads_and(w_ok);  // also orders the previous chunk's reads of `fac`
    if (!ok) break;
    // per-point factors from the prefetched angles: (cos, sin of theta_q / 2, Jx, Jy), (Jt, .)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int e = tid + j * WG_THREADS;
      if (e < ppc * n) {
        const float4 tq = pf.tj[j];
        float sn, cs;
        sincosf(0.5f * tq.x, &sn, &cs);
        const int pl = e / n, q = e % n;
        const bool valid = p0 + pl < a.npts[set];  // rows past the end of the set contribute zero
        fac[(pl * n + q) * 2] = valid ? make_float4(cs, sn, tq.y, tq.z) : make_float4(0.f, 0.f, 0.f, 0.f);
        fac[(pl * n + q) * 2 + 1] = valid ? make_float4(tq.w, 1.f, 0.f, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    // B: costate rows of the chunk (prefetched) -> (o, row) core layout, TF32 hi/lo
    {
      float* Bhi = reinterpret_cast<float*>(sB);
      float* Blo = reinterpret_cast<float*>(sB + bbytes);
#pragma unroll
      for (int g4 = 0; g4 < KC / 4; ++g4) {
        float4 h4, l4;
        qptc::split_tf32(pf.lam[4 * g4], h4.x, l4.x);
        qptc::split_tf32(pf.lam[4 * g4 + 1], h4.y, l4.y);
        qptc::split_tf32(pf.lam[4 * g4 + 2], h4.z, l4.z);
        qptc::split_tf32(pf.lam[4 * g4 + 3], h4.w, l4.w);
        const uint32_t off = core_off(tid, g4 * 4) / 4;
        *reinterpret_cast<float4*>(Bhi + off) = h4;
        *reinterpret_cast<float4*>(Blo + off) = l4;
      }
    }
    __syncthreads();  // fac visible
    // next chunk's global loads are in flight while this chunk is generated and multiplied
    if (kc + 1 < kc1) wg_prefetch(a, kc + 1, tid, o, pf);
    float* Ahi = reinterpret_cast<float*>(sA);
    float* Alo = reinterpret_cast<float*>(sA + abytes);
    float av[KC / 2];  // this thread's half of the row: K indices 16 * ahalf .. + 15
    if (set == 0) {
#pragma unroll
      for (int pi = 0; pi < 4; ++pi) {
        const int pl = ahalf * 4 + pi;
        float P = 1.f, D0 = 0.f, D1 = 0.f, D2 = 0.f;
        for (int q = 0; q < n; ++q) {
          const float4 f0 = fac[(pl * n + q) * 2], f1 = fac[(pl * n + q) * 2 + 1];
          const bool bit = (krow >> (n - 1 - q)) & 1;
          const float f = bit ? f0.y : f0.x, d = bit ? 0.5f * f0.x : -0.5f * f0.y;
          D0 = D0 * f + P * d * f0.z;
          D1 = D1 * f + P * d * f0.w;
          D2 = D2 * f + P * d * f1.x;
          P *= f;
        }
        av[4 * pi] = P; av[4 * pi + 1] = D0; av[4 * pi + 2] = D1; av[4 * pi + 3] = D2;
      }
    } else {
#pragma unroll
      for (int pi = 0; pi < 16; ++pi) {
        const int pl = ahalf * 16 + pi;
        float P = 1.f;
        for (int q = 0; q < n; ++q) {
          const float4 f0 = fac[(pl * n + q) * 2];
          P *= ((krow >> (n - 1 - q)) & 1) ? f0.y : f0.x;
        }
        av[pi] = P;
      }
    }
#pragma unroll
    for (int g4 = 0; g4 < KC / 8; ++g4) {
      float4 h4, l4;
      qptc::split_tf32(av[4 * g4], h4.x, l4.x);
      qptc::split_tf32(av[4 * g4 + 1], h4.y, l4.y);
      qptc::split_tf32(av[4 * g4 + 2], h4.z, l4.z);
      qptc::split_tf32(av[4 * g4 + 3], h4.w, l4.w);
      const uint32_t off = core_off(arow, ahalf * (KC / 2) + g4 * 4) / 4;
      *reinterpret_cast<float4*>(Ahi + off) = h4;
      *reinterpret_cast<float4*>(Alo + off) = l4;
    }
    qptc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      qptc::fence_after();
      const uint32_t sa = qptc::smem_u32(sA), sb = qptc::smem_u32(sB);
#pragma unroll
      for (int ks = 0; ks < KC / 8; ++ks) {
        const uint64_t ah = qptc::desc_kmajor(sa + ks * 256, 128, (KC / 4) * 128);
        const uint64_t al = qptc::desc_kmajor(sa + abytes + ks * 256, 128, (KC / 4) * 128);
        const uint64_t bh = qptc::desc_kmajor(sb + ks * 256, 128, (KC / 4) * 128);
        const uint64_t bl = qptc::desc_kmajor(sb + bbytes + ks * 256, 128, (KC / 4) * 128);
        qptc::mma_tf32(tmem, ah, bh, id, (kc > kc0 || ks > 0) ? 1u : 0u);
        qptc::mma_tf32(tmem, ah, bl, id, 1u);
        qptc::mma_tf32(tmem, al, bh, id, 1u);
      }
      qptc::commit(&bars[st]);
    }
  }
  // epilogue: 128 x 256 partial tile; warps w and w + 4 read the same lanes, column halves
  const int lrow = (warp & 3) * 32 + (tid & 31), chalf = warp >> 2;
  float* outp = a.part + ((int64_t)blockIdx.y * dim + mt * TM + lrow) * (2 * dim) + nt * nch + chalf * 128;
  if (ok && it > 0) {
    ok = __syncthreads_and(qptc::mbar_wait(&bars[(it - 1) & 1], ((it - 1) >> 1) & 1));
    if (ok) {
      qptc::fence_after();
      float v[32];
      for (int c0 = 0; c0 < 128; c0 += 32) {
        qptc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + chalf * 128 + c0, v);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          reinterpret_cast<float4*>(outp + c0)[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
      }
    }
  } else if (ok) {
    for (int c0 = 0; c0 < 128; c0 += 4) *reinterpret_cast<float4*>(outp + c0) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.status, 6);
    if (it >= 1) qptc::mbar_wait(&bars[(it - 1) & 1], ((it - 1) >> 1) & 1);
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, 256);
}

}  // namespace qpd
