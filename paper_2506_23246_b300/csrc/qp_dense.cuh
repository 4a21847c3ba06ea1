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
#include <cuda_runtime.h>

#include "qp_circuit.cuh"
#include "qp_common.h"
#include "qp_tc.cuh"

namespace qpd {

constexpr int KC = 32;        // K (basis index) elements per chunk
constexpr int TM = 128;       // rows per tile (tensor-memory lanes)

__host__ __device__ inline int n_cols_chunk(int n) { return (2 << n) < 256 ? (2 << n) : 256; }

// Byte offset of element (row r, k-in-chunk t) in a K-major, no-swizzle operand block whose
// 8-row groups hold KC/4 core matrices of 8 x 16 bytes.
__host__ __device__ inline uint32_t core_off(int r, int t) {
  return (uint32_t)((r >> 3) * (KC / 4) * 128 + (t >> 2) * 128 + (r & 7) * 16 + (t & 3) * 4);
}

// ------------------------------------------------------------------------- unitary build
struct BuildArgs {
  const float* params;
  int64_t circ_off;
  int32_t n, L, ansatz, enc;
  float* W;        // [ncc][nkc][2 (hi, lo)][nch x KC] tiled operand blocks
  double2* U;      // [2^n][2^n] fused unitary U' (row j, column k), FP64, or null
};

__device__ inline double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One block per basis column k: |k> through all layers (gates and CNOT rings) in FP64.
__global__ void dense_build_kernel(BuildArgs a) {
  extern __shared__ __align__(16) double2 col[];
  __shared__ double2 g[4];
  const int n = a.n, dim = 1 << n, k = blockIdx.x;
  for (int j = threadIdx.x; j < dim; j += blockDim.x) col[j] = make_double2(j == k ? 1.0 : 0.0, 0.0);
  __syncthreads();
  const int kp = a.ansatz == 0 ? 2 : 3;
  for (int l = 0; l < a.L; ++l) {
    for (int q = 0; q < n; ++q) {
      if (threadIdx.x == 0) {
        const float* p = a.params + a.circ_off + ((int64_t)l * n + q) * kp;
        double c0, s0;
        double2 u00, u01, u10, u11;
        if (a.ansatz == 0) {  // RZ(b) RY(a)
          double ca, sa, cb, sb;
          sincos(0.5 * (double)p[0], &sa, &ca);
          sincos(0.5 * (double)p[1], &sb, &cb);
          u00 = make_double2(cb * ca, -sb * ca);
          u01 = make_double2(-cb * sa, sb * sa);
          u10 = make_double2(cb * sa, sb * sa);
          u11 = make_double2(cb * ca, sb * ca);
        } else {              // RZ(g) RY(b) RZ(a)
          double cb, sb;
          sincos(0.5 * (double)p[1], &sb, &cb);
          const double ap = 0.5 * ((double)p[0] + (double)p[2]), am = 0.5 * ((double)p[0] - (double)p[2]);
          double cp, sp, cm, sm;
          sincos(ap, &sp, &cp);
          sincos(am, &sm, &cm);
          u00 = make_double2(cp * cb, -sp * cb);
          u01 = make_double2(-cm * sb, -sm * sb);
          u10 = make_double2(cm * sb, -sm * sb);
          u11 = make_double2(cp * cb, sp * cb);
        }
        (void)c0; (void)s0;
        g[0] = u00; g[1] = u01; g[2] = u10; g[3] = u11;
      }
      __syncthreads();
      const int bit = 1 << (n - 1 - q);
      for (int i = threadIdx.x; i < dim / 2; i += blockDim.x) {
        const int k0 = ((i & ~(bit - 1)) << 1) | (i & (bit - 1));
        const int k1 = k0 | bit;
        const double2 x = col[k0], y = col[k1];
        const double2 a0 = zmul(g[0], x), a1 = zmul(g[1], y), b0 = zmul(g[2], x), b1 = zmul(g[3], y);
        col[k0] = make_double2(a0.x + a1.x, a0.y + a1.y);
        col[k1] = make_double2(b0.x + b1.x, b0.y + b1.y);
      }
      __syncthreads();
    }
    if (a.ansatz != 3 && n > 1) {
      const int r = a.ansatz == 2 ? 1 + (l % (n - 1)) : 1;
      for (int i = 0; i < n; ++i) {
        const int bc = 1 << (n - 1 - i), bt = 1 << (n - 1 - (i + r) % n);
        for (int j = threadIdx.x; j < dim; j += blockDim.x) {
          if ((j & bc) && !(j & bt)) {
            const double2 t = col[j];
            col[j] = col[j | bt];
            col[j | bt] = t;
          }
        }
        __syncthreads();
      }
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
    const double2 v = zmul(col[j], ph);
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
      const int c = o / nch, r = o % nch;
      float* blk = a.W + ((int64_t)(c * nkc + kc) * 2) * (nch * KC);
      blk[core_off(r, t) / 4] = hi;
      blk[nch * KC + core_off(r, t) / 4] = lo;
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
};

// Smem: 2 stages x (A hi, A lo: 128 x KC fp32; W hi, W lo: nch x KC fp32) + barriers.
__host__ __device__ inline int gemm_smem_bytes(int n) {
  const int nch = n_cols_chunk(n);
  return 2 * (2 * TM * KC * 4 + 2 * nch * KC * 4) + 128;
}

__global__ void __launch_bounds__(128, 1) dense_fwd_gemm_kernel(GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int n = a.n, dim = 1 << n;
  const int nch = n_cols_chunk(n), ncc = (2 * dim) / nch, nkc = dim / KC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int abytes = TM * KC * 4, wbytes = nch * KC * 4;
  const int stage_bytes = 2 * abytes + 2 * wbytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);  // w_full[2], mma_done[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage_bytes + 64);
  const uint32_t tcols = nch * 2 <= 32 ? 32 : (nch * 2 <= 64 ? 64 : (nch * 2 <= 128 ? 128 : (nch * 2 <= 256 ? 256 : 512)));
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
    for (int b = 0; b < low; ++b) {
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
        }
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
        float* Ahi = reinterpret_cast<float*>(sA);
        float* Alo = reinterpret_cast<float*>(sA + abytes);
        const int r = tid;  // tile row owned by this thread
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
        qptc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          ok = qptc::mbar_wait(&bars[st], (it >> 1) & 1);
          if (ok) {
            qptc::fence_after();
            const uint32_t sa = qptc::smem_u32(sA), sw = qptc::smem_u32(sW);
            const uint32_t dt = tmem + cbuf * (tcols / 2);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
              const uint64_t ah = qptc::desc_kmajor(sa + ks * 256, 128, (KC / 4) * 128);
              const uint64_t al = qptc::desc_kmajor(sa + abytes + ks * 256, 128, (KC / 4) * 128);
              const uint64_t wh = qptc::desc_kmajor(sw + ks * 256, 128, (KC / 4) * 128);
              const uint64_t wl = qptc::desc_kmajor(sw + wbytes + ks * 256, 128, (KC / 4) * 128);
              qptc::mma_tf32(dt, ah, wh, id, (kc > 0 || ks > 0) ? 1u : 0u);
              qptc::mma_tf32(dt, ah, wl, id, 1u);
              qptc::mma_tf32(dt, al, wh, id, 1u);
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
            float v[32];
            for (int c0 = 0; c0 < nch; c0 += 32) {
              qptc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + pend_buf * (tcols / 2) + c0, v);
              if (pp < a.npts) {
                float4* dst = reinterpret_cast<float4*>(a.phi + ((a.pt_base + pp) * 4 + s) * dim) +
                              (pending * nch + c0) / 4;
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
      float v[32];
      for (int c0 = 0; c0 < nch; c0 += 32) {
        qptc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + pend_buf * (tcols / 2) + c0, v);
        if (pp < a.npts) {
          float4* dst = reinterpret_cast<float4*>(a.phi + ((a.pt_base + pp) * 4 + s) * dim) +
                        (pending * nch + c0) / 4;
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
};

__global__ void dense_point_kernel(PointArgs a) {
  extern __shared__ __align__(16) unsigned char psh[];
  const int n = a.n, dim = 1 << n, m = a.m;
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
  for (int64_t gq = wg; gq < total; gq += nw) {
    int set = 0;
    int64_t li = gq;
    if (li >= a.npts[0]) { li -= a.npts[0]; set = 1; if (li >= a.npts[1]) { li -= a.npts[1]; set = 2; } }
    const int nv = set == 0 ? 4 : 1;
    float2* ph = a.phi + (a.pt_base[set] + li) * 4 * dim;
    float z[QP_MAXQ], dz[3][QP_MAXQ];
#pragma unroll
    for (int i = 0; i < QP_MAXQ; ++i) { z[i] = 0.f; dz[0][i] = dz[1][i] = dz[2][i] = 0.f; }
    for (int k = lane; k < dim; k += 32) {
      const float2 f0 = ph[k];
      const float pr = f0.x * f0.x + f0.y * f0.y;
      float q[3] = {0.f, 0.f, 0.f};
      if (nv == 4) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float2 fd = ph[(1 + d) * dim + k];
          q[d] = 2.f * (fd.x * f0.x + fd.y * f0.y);
        }
      }
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i)
        if (i < m) {
          const float sg = ((k >> (n - 1 - i)) & 1) ? -1.f : 1.f;
          z[i] += sg * pr;
#pragma unroll
          for (int d = 0; d < 3; ++d) dz[d][i] += sg * q[d];
        }
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
    qpk::point_loss(a.pb, set, li, a.npts[set], a.counts, xp[0], xp[1], f, D, true, lane == 0, sloss, g, gD);
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
        for (int i = 0; i < m; ++i)
          atomicAdd(&hacc[c * m + i], g[c] * z[i] + gD[c][0] * dz[0][i] + gD[c][1] * dz[1][i] + gD[c][2] * dz[2][i]);
        atomicAdd(&hacc[3 * m + c], g[c]);
      }
    }
    for (int k = lane; k < dim; k += 32) {
      float O = 0.f, Od[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < QP_MAXQ; ++i)
        if (i < m) {
          const float sg = ((k >> (n - 1 - i)) & 1) ? -1.f : 1.f;
          O += sg * zb[i];
#pragma unroll
          for (int d = 0; d < 3; ++d) Od[d] += sg * zbd[d][i];
        }
      const float2 f0 = ph[k];
      float2 lam = make_float2(O * f0.x, O * f0.y);
      if (nv == 4) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float2 fd = ph[(1 + d) * dim + k];
          lam.x += Od[d] * fd.x;
          lam.y += Od[d] * fd.y;
          ph[(1 + d) * dim + k] = make_float2(Od[d] * f0.x, Od[d] * f0.y);
        }
      }
      ph[k] = lam;
    }
  }
  __syncthreads();
  double* bl = a.blk_loss + (int64_t)blockIdx.x * a.loss_stride;
  for (int i = threadIdx.x; i < QP_NLP + nt; i += blockDim.x) bl[i] = sloss[i];
  float* bg = a.blk_grad + (int64_t)blockIdx.x * a.grad_stride;
  for (int i = threadIdx.x; i < a.nE; i += blockDim.x) bg[i] = 0.f;
  for (int i = threadIdx.x; i < 3 * m + 3; i += blockDim.x) bg[a.nE + i] = hacc[i];
}

// ------------------------------------------------------------------------- weight-gradient GEMM
// G_part[chunk][k][o] = sum over the chunk's (point, vector) rows of R_s[k] * Lambda_s[o]:
// M = 128 basis indices k, N = 256 costate components o = (amp, re|im), K = (point, vector).
// R is regenerated from the angles; Lambda is read from the costate buffer.
struct WgArgs {
  const float* thetaJ;
  const float2* lam;          // [P][4][dim]
  float* part;                // [nchunks][dim][2 dim]
  int32_t n;
  int64_t npts[3], pt_base[3];
  int64_t rows_total;         // sum over sets of points * vectors, in K order
  int32_t nchunks;            // point chunks (grid.y)
  int32_t* status;
};

__host__ __device__ inline int wg_smem_bytes() { return 2 * (2 * TM * KC * 4 + 2 * 256 * KC * 4) + 128 + 32 * 40 * 4; }

// Map K row index (concatenated sets: colloc rows are (point, vector) with vector fastest)
__device__ __forceinline__ void wg_row(const WgArgs& a, int64_t r, int& set, int64_t& p, int& s) {
  const int64_t r0 = a.npts[0] * 4;
  if (r < r0) { set = 0; p = r >> 2; s = (int)(r & 3); return; }
  r -= r0;
  if (r < a.npts[1]) { set = 1; p = r; s = 0; return; }
  set = 2; p = r - a.npts[1]; s = 0;
}

__global__ void __launch_bounds__(128, 1) dense_wgrad_gemm_kernel(WgArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int n = a.n, dim = 1 << n;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = blockIdx.x % (dim / TM), nt = blockIdx.x / (dim / TM);
  const int nch = 256;
  const int abytes = TM * KC * 4, bbytes = nch * KC * 4;
  const int stage_bytes = 2 * abytes + 2 * bbytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);  // mma_done[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * stage_bytes + 64);
  float* fac = reinterpret_cast<float*>(sm + 2 * stage_bytes + 128);   // [32 rows][n][4]
  if (warp == 0) qptc::tmem_alloc(tslot, 256);
  if (tid == 0) { qptc::mbar_init(&bars[0], 1); qptc::mbar_init(&bars[1], 1); }
  qptc::fence_before();
  __syncthreads();
  qptc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = qptc::idesc(2, TM, nch);
  const int64_t nkc_total = (a.rows_total + KC - 1) / KC;
  const int64_t per = (nkc_total + a.nchunks - 1) / a.nchunks;
  const int64_t kc0 = blockIdx.y * per;
  const int64_t kc1 = kc0 + per < nkc_total ? kc0 + per : nkc_total;
  const int krow = mt * TM + tid;  // basis index owned by this thread in the A operand
  bool ok = true;
  uint32_t it = 0;
  for (int64_t kc = kc0; kc < kc1 && ok; ++kc, ++it) {
    const uint32_t st = it & 1;
    unsigned char* sA = sm + st * stage_bytes;
    unsigned char* sB = sA + 2 * abytes;
    bool w_ok = true;
    if (it >= 2) w_ok = qptc::mbar_wait(&bars[st], ((it - 2) >> 1) & 1);
    ok = __syncthreads_and(w_ok);
    if (!ok) break;
    // per-row factors of the chunk: cos, sin of theta_q/2 and the row's Jacobian direction
    for (int e = tid; e < KC * n; e += blockDim.x) {
      const int t = e / n, q = e % n;
      const int64_t r = kc * KC + t;
      float4 v = make_float4(1.f, 0.f, 0.f, 0.f);  // rows past the end contribute zero
      if (r < a.rows_total) {
        int set, s;
        int64_t p;
        wg_row(a, r, set, p, s);
        const float4 tq = reinterpret_cast<const float4*>(a.thetaJ)[(a.pt_base[set] + p) * n + q];
        float sn, cs;
        sincosf(0.5f * tq.x, &sn, &cs);
        v = make_float4(cs, sn, s == 1 ? tq.y : (s == 2 ? tq.z : tq.w), (float)s);
      } else {
        v = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      reinterpret_cast<float4*>(fac)[t * n + q] = v;
    }
    __syncthreads();
    // A: R_s[krow] for the 32 rows of the chunk (product rule for the tangents)
    {
      float* Ahi = reinterpret_cast<float*>(sA);
      float* Alo = reinterpret_cast<float*>(sA + abytes);
#pragma unroll
      for (int g4 = 0; g4 < KC / 4; ++g4) {
        float4 h4, l4;
        float* hv = &h4.x;
        float* lv = &l4.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int t = g4 * 4 + e;
          const float4* ft = reinterpret_cast<const float4*>(fac) + t * n;
          float P = 1.f, Pd = 0.f;
          const int s = (int)ft[0].w;
          for (int q = 0; q < n; ++q) {
            const float4 fq = ft[q];
            const bool bit = (krow >> (n - 1 - q)) & 1;
            const float f = bit ? fq.y : fq.x, d = bit ? 0.5f * fq.x : -0.5f * fq.y;
            Pd = Pd * f + P * d * fq.z;
            P *= f;
          }
          qptc::split_tf32(s == 0 ? P : Pd, hv[e], lv[e]);
        }
        const uint32_t off = core_off(tid, g4 * 4) / 4;
        *reinterpret_cast<float4*>(Ahi + off) = h4;
        *reinterpret_cast<float4*>(Alo + off) = l4;
      }
    }
    // B: Lambda rows -> (o, row) core layout; thread handles o = tid and tid + 128
    {
      float* Bhi = reinterpret_cast<float*>(sB);
      float* Blo = reinterpret_cast<float*>(sB + bbytes);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int orow = tid + half * 128;
        const int o = nt * nch + orow;
#pragma unroll
        for (int g4 = 0; g4 < KC / 4; ++g4) {
          float4 h4, l4;
          float* hv = &h4.x;
          float* lv = &l4.x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int64_t r = kc * KC + g4 * 4 + e;
            float v = 0.f;
            if (r < a.rows_total) {
              int set, s;
              int64_t p;
              wg_row(a, r, set, p, s);
              v = reinterpret_cast<const float*>(a.lam + ((a.pt_base[set] + p) * 4 + s) * dim)[o];
            }
            qptc::split_tf32(v, hv[e], lv[e]);
          }
          const uint32_t off = core_off(orow, g4 * 4) / 4;
          *reinterpret_cast<float4*>(Bhi + off) = h4;
          *reinterpret_cast<float4*>(Blo + off) = l4;
        }
      }
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
    __syncthreads();
  }
  // epilogue: 128 x 256 partial tile
  float* outp = a.part + ((int64_t)blockIdx.y * dim + mt * TM + tid) * (2 * dim) + nt * nch;
  if (ok && it > 0) {
    ok = __syncthreads_and(qptc::mbar_wait(&bars[(it - 1) & 1], ((it - 1) >> 1) & 1));
    if (ok) {
      qptc::fence_after();
      float v[32];
      for (int c0 = 0; c0 < nch; c0 += 32) {
        qptc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          reinterpret_cast<float4*>(outp + c0)[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
      }
    }
  } else if (ok) {
    for (int c0 = 0; c0 < nch; c0 += 4) *reinterpret_cast<float4*>(outp + c0) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.status, 6);
    if (it >= 1) qptc::mbar_wait(&bars[(it - 1) & 1], ((it - 1) >> 1) & 1);
  }
  qptc::fence_before();
  __syncthreads();
  if (warp == 0) qptc::tmem_dealloc(tmem, 256);
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
  float* eout;          // blk_grad block 0: E[(l n + q) * 3 + P]
};

__global__ void dense_gsum_kernel(SweepArgs a) {
  const int dim = 1 << a.n;
  const int64_t tot = (int64_t)dim * dim;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / dim, j = e % dim;
    double re = 0.0, im = 0.0;
    for (int c = 0; c < a.nchunks; ++c) {
      const float* r = a.part + ((int64_t)c * dim + k) * (2 * dim);
      re += r[2 * j];
      im -= r[2 * j + 1];
    }
    a.G[e] = make_float2((float)re, (float)im);
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

// One block: Y <- C^dag Y C for each ring, E_P(l,q) = Im Tr(P_q Y), Y <- R^dag Y R, l = L-1..0.
__global__ void dense_sweep_kernel(SweepArgs a) {
  const int n = a.n, dim = 1 << n;
  float2* Y = a.Y;
  __shared__ float red[3][32];
  __shared__ double2 gm[4];
  const int kp = a.ansatz == 0 ? 2 : 3;
  for (int l = a.L - 1; l >= 0; --l) {
    if (a.ansatz != 3 && n > 1) {
      const int r = a.ansatz == 2 ? 1 + (l % (n - 1)) : 1;
      // undo the ring: CNOTs in reverse order, each a swap of rows and of columns
      for (int i = n - 1; i >= 0; --i) {
        const int bc = 1 << (n - 1 - i), bt = 1 << (n - 1 - (i + r) % n);
        for (int64_t e = threadIdx.x; e < (int64_t)dim * dim; e += blockDim.x) {
          const int row = (int)(e / dim), col = (int)(e % dim);
          if ((row & bc) && !(row & bt)) {
            const float2 t = Y[e];
            Y[e] = Y[(int64_t)(row | bt) * dim + col];
            Y[(int64_t)(row | bt) * dim + col] = t;
          }
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)dim * dim; e += blockDim.x) {
          const int row = (int)(e / dim), col = (int)(e % dim);
          if ((col & bc) && !(col & bt)) {
            const float2 t = Y[e];
            Y[e] = Y[(int64_t)row * dim + (col | bt)];
            Y[(int64_t)row * dim + (col | bt)] = t;
          }
        }
        __syncthreads();
      }
    }
    for (int q = 0; q < n; ++q) {
      const int bit = 1 << (n - 1 - q);
      // E_X = Im sum_a Y[a^q][a]; E_Y = Im sum_a P_{a,a^q} Y[a^q][a]; E_Z = Im sum_a z_a Y[a][a]
      float ex = 0.f, ey = 0.f, ez = 0.f;
      for (int ai = threadIdx.x; ai < dim; ai += blockDim.x) {
        const float2 y1 = Y[(int64_t)(ai ^ bit) * dim + ai];
        const float2 yd = Y[(int64_t)ai * dim + ai];
        ex += y1.y;
        // P_{a,a^q} = -i (bit 0) or +i (bit 1): Im(-i y) = -y.x, Im(i y) = y.x
        ey += (ai & bit) ? y1.x : -y1.x;
        ez += (ai & bit) ? -yd.y : yd.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ex += __shfl_xor_sync(0xffffffffu, ex, o);
        ey += __shfl_xor_sync(0xffffffffu, ey, o);
        ez += __shfl_xor_sync(0xffffffffu, ez, o);
      }
      if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = ex; red[1][threadIdx.x >> 5] = ey; red[2][threadIdx.x >> 5] = ez; }
      if (threadIdx.x == 0) {
        const float* p = a.params + a.circ_off + ((int64_t)l * n + q) * kp;
        double2 u00, u01, u10, u11;
        if (a.ansatz == 0) {
          double ca, sa, cb, sb;
          sincos(0.5 * (double)p[0], &sa, &ca);
          sincos(0.5 * (double)p[1], &sb, &cb);
          u00 = make_double2(cb * ca, -sb * ca); u01 = make_double2(-cb * sa, sb * sa);
          u10 = make_double2(cb * sa, sb * sa); u11 = make_double2(cb * ca, sb * ca);
        } else {
          double cb, sb;
          sincos(0.5 * (double)p[1], &sb, &cb);
          const double ap = 0.5 * ((double)p[0] + (double)p[2]), am = 0.5 * ((double)p[0] - (double)p[2]);
          double cp, sp, cm, smm;
          sincos(ap, &sp, &cp);
          sincos(am, &smm, &cm);
          u00 = make_double2(cp * cb, -sp * cb); u01 = make_double2(-cm * sb, -smm * sb);
          u10 = make_double2(cm * sb, -smm * sb); u11 = make_double2(cp * cb, sp * cb);
        }
        gm[0] = u00; gm[1] = u01; gm[2] = u10; gm[3] = u11;
      }
      __syncthreads();
      if (threadIdx.x < 3) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        a.eout[(l * n + q) * 3 + threadIdx.x] = s;
      }
      // Y <- U^dag Y U on qubit q (rows by U^dag, columns by U)
      const float2 u00 = make_float2((float)gm[0].x, (float)gm[0].y), u01 = make_float2((float)gm[1].x, (float)gm[1].y);
      const float2 u10 = make_float2((float)gm[2].x, (float)gm[2].y), u11 = make_float2((float)gm[3].x, (float)gm[3].y);
      for (int64_t e = threadIdx.x; e < (int64_t)dim * dim / 2; e += blockDim.x) {
        const int col = (int)(e % dim), ri = (int)(e / dim);
        const int r0 = ((ri & ~(bit - 1)) << 1) | (ri & (bit - 1)), r1 = r0 | bit;
        const float2 x = Y[(int64_t)r0 * dim + col], y = Y[(int64_t)r1 * dim + col];
        // rows: U^dag = [[conj u00, conj u10], [conj u01, conj u11]]
        Y[(int64_t)r0 * dim + col] = make_float2(u00.x * x.x + u00.y * x.y + u10.x * y.x + u10.y * y.y,
                                                 u00.x * x.y - u00.y * x.x + u10.x * y.y - u10.y * y.x);
        Y[(int64_t)r1 * dim + col] = make_float2(u01.x * x.x + u01.y * x.y + u11.x * y.x + u11.y * y.y,
                                                 u01.x * x.y - u01.y * x.x + u11.x * y.y - u11.y * y.x);
      }
      __syncthreads();
      for (int64_t e = threadIdx.x; e < (int64_t)dim * dim / 2; e += blockDim.x) {
        const int row = (int)(e / (dim / 2)), ci = (int)(e % (dim / 2));
        const int c0 = ((ci & ~(bit - 1)) << 1) | (ci & (bit - 1)), c1 = c0 | bit;
        const float2 x = Y[(int64_t)row * dim + c0], y = Y[(int64_t)row * dim + c1];
        // columns: (Y U)[., c0] = Y[.,c0] u00 + Y[.,c1] u10 ; (Y U)[., c1] = Y[.,c0] u01 + Y[.,c1] u11
        Y[(int64_t)row * dim + c0] = make_float2(x.x * u00.x - x.y * u00.y + y.x * u10.x - y.y * u10.y,
                                                 x.x * u00.y + x.y * u00.x + y.x * u10.y + y.y * u10.x);
        Y[(int64_t)row * dim + c1] = make_float2(x.x * u01.x - x.y * u01.y + y.x * u11.x - y.y * u11.y,
                                                 x.x * u01.y + x.y * u01.x + y.x * u11.y + y.y * u11.x);
      }
      __syncthreads();
    }
  }
}

}  // namespace qpd
