// qp_api.cu -- the C-ABI of libqpinn.so (declared in include/qpinn.h): plan creation and
// validation, workspace carving and the launch sequence of one forward or loss+gradient call.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cublas_v2.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>
#include <new>

#include "../../include/qpinn.h"
#include "qp_aux.cuh"
#include "qp_premap_tc.cuh"
#include "qp_circuit.cuh"
#include "qp_common.h"
#include "qp_dense.cuh"
#include "qp_fused.cuh"
#include "qp_mlp.cuh"
#include "qp_mu.cuh"
#include "qp_wgrad.cuh"

extern "C" int qp_build_sched(int n, int L, int ansatz, QPSched* out);

struct qp_plan {
  qp_circuit c;
  qp_problem p;
  int32_t path;
  QPSched sched;
  int device = 0, sm_count = 0;
  // sharding of the current loss call (qp_batch norm_* fields; zeros: unsharded)
  int64_t cur_norm[3] = {0, 0, 0}, cur_norm_diel = 0, cur_colloc_off = 0;
  int warps_grad = 0, blocks_grad = 0, warps_fwd = 0, blocks_fwd = 0;
  int smem_grad = 0, smem_fwd = 0, sstride_grad = 0, sstride_fwd = 0;
  int nwblk = 0, wtile = 0, smem_wgrad = 0, smem_premap = 0, smem_premap4 = 0;
  int wblk = 0;   // premap weight-gradient slots written by the last premap backward (<= nwblk)
  bool swc_big = false;   // the one-launch sweep runs as a 16-CTA cluster
  bool pg_ok = false;     // RFF + MLP premap with F = 64, H = 32: the GEMM-formulated kernels
  bool deep = false;      // RFF + MLP premap of another depth or width: the layer-by-layer kernels
  int32_t operands = QP_OPERANDS_FP16_PAIRS;   // forward contraction outside the fused kernel
  int64_t n_params = 0, circ_off = 0, head_off = 0, mlp_off = 0, mlp_count = 0, nfixed = 0;
  int32_t nE = 0;   // gate-gradient partial sums per block: 3 n L Pauli sums + L CRZ sums
  uint32_t wait_limit = 0;   // pipeline-wait polls of the fused forward (0: the kernel's default)
  // multi-instance launch (qp_batch_step): the tuned shape of the last batch this plan was tuned
  // in, keyed by that batch's signature (0: none)
  uint64_t mt_sig = 0;
  int32_t mt_warps = 0, mt_items = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int32_t last_launches = 0;
  cudaStream_t last_stream = nullptr;
  // device status word of the last compute call: the workspace's, or the fixed array's after
  // qp_forward_noalloc (null before the first call)
  const int32_t* last_status = nullptr;
  // profiling events per measured kernel (qp_set_profile_events): [0] statevector kernel or
  // forward contraction, [1] weight-gradient contraction, [2] back-projection mu
  cudaEvent_t prof_start[3] = {nullptr, nullptr, nullptr}, prof_stop[3] = {nullptr, nullptr, nullptr};
  // tensor-core path: a side stream for the unitary build, which runs beside the premap (forked
  // from and joined back into the call's stream within the call)
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // layer-by-layer premap: the library GEMM handle of its contractions and the compute type
  // that handle accepted (FP32 emulated on the tensor cores, else plain FP32)
  cublasHandle_t blas = nullptr;
  cublasComputeType_t blas_ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
  ~qp_plan() {
    if (blas) cublasDestroy(blas);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (aux) cudaStreamDestroy(aux);
  }
};

namespace {

constexpr int kMaxWarps = 12;
constexpr size_t kBlasWorkspace = size_t(32) << 20;   // library GEMM scratch of a deep-premap call

// Fixed RFF frequencies: Omega [F][3], or [F][6] with the periodic input map.
int64_t omega_count(const qp_circuit& c) {
  return c.premap == QP_PREMAP_RFF_MLP ? (c.periodic ? 6LL : 3LL) * c.rff_freqs : 0;
}

int64_t premap_count(const qp_circuit& c) {
  if (c.premap != QP_PREMAP_RFF_MLP) return 0;
  int64_t cnt = omega_count(c) + (c.periodic ? 1 : 0);
  int64_t in = 2LL * c.rff_freqs;
  for (int l = 0; l < c.mlp_depth; ++l) { cnt += (int64_t)c.mlp_width * in + c.mlp_width; in = c.mlp_width; }
  cnt += (int64_t)c.n_qubits * in + c.n_qubits;
  return cnt;
}

int geo_lb(int n) { return n <= 3 ? n : (n <= 8 ? 3 : n - 5); }
int geo_ppw(int n) { return 32 >> (n - geo_lb(n)); }

// Dynamic shared-memory allowance of a kernel. The attribute belongs to the function, not to a
// plan, so plans only ever raise it: a plan created later with a smaller need must not shrink
// the allowance an earlier plan's launches rely on.
static std::mutex g_attr_mu;
// The weight-gradient kernel compiled for n qubits (7 .. 10; plans of fewer qubits never launch
// it and take the 7-qubit form for their shared-memory limit).
template <bool H16>
static const void* wgrad_kernel(int n) {
  switch (n) {
    case 10: return (const void*)qpd::dense_wgrad_gemm_kernel<H16, 10>;
    case 9: return (const void*)qpd::dense_wgrad_gemm_kernel<H16, 9>;
    case 8: return (const void*)qpd::dense_wgrad_gemm_kernel<H16, 8>;
    default: return (const void*)qpd::dense_wgrad_gemm_kernel<H16, 7>;
  }
}

static cudaError_t raise_smem_limit(const void* fn, cudaFuncAttribute attr, int bytes) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(fn, attr, bytes);
}

struct WsLayout {
  size_t status, gates, cmat, cenc, crz, crz64, thetaJ, dthetaJ, d1, d2, u1, blk_loss, blk_grad, wpart;
  size_t mact, mcot;   // layer-by-layer premap: hidden activations, two cotangent buffers
  size_t sxb, sF, sgs, sge, spart;   // symmetry penalty: set-2 points, fields, cotangents, sums
  size_t mtg;                        // periodic map: FP64 sum of the learned period's gradient
  size_t desc;                       // multi-instance launch: the instance's argument block
  size_t mx0, blasws;                // layer-by-layer premap: RFF features [P][4][2F], GEMM scratch
  size_t mwt, mdw;                   // ... aligned copies of the layers' weights, per-chunk dW
  size_t dW, dphi, dU, dG, dY, dpart, dWT, dmu, dW16, dcs, dgs, dgates, total;
};

// Rows of (point, vector) accumulated per weight-gradient chunk (bounds the FP32 tensor-core
// accumulation length; chunks are summed in FP64).
// Rows accumulated in tensor memory before a flush. The tensor core adds each instruction's
// products into the FP32 accumulator with a truncating alignment (about one accumulator ulp
// per instruction, not averaging out), and the three FP16-pair products of a 16-row step go to
// the same accumulator: 512 rows (96 instructions) keep the full-size weight gradient within
// ~4e-6 of the FP32 SIMT path; 4096 rows reached 2e-5.
// 3xTF32 operands take two instructions per product of a 16-row step (K = 8 each) where FP16
// pairs take one, so their accumulator is flushed every 256 rows: the same number of
// truncating instructions per flush.
int64_t wg_rows_per_chunk(const qp_plan* pl) {
  const bool h16 = (pl->c.n_qubits <= 8) || pl->operands == QP_OPERANDS_FP16_PAIRS;
  return h16 ? 512 : 256;
}

// Weight-gradient launch geometry for `nkc` 16-row steps: tiles of min(256, 2^n) basis
// indices x 256 components; the tiles' steps as one tile-major sequence split into `grid`
// balanced ranges (persistent CTAs, one per SM; a range meets at most two tiles); steps per
// flush (at most wg_rows_per_chunk rows); partial slots per tile: the most CTAs any tile meets.
struct WgGeom {
  int tiles, grid, fl;
  int64_t nslots;
};
static int wg_tiles(const qp_plan* pl) {
  const int n = pl->c.n_qubits, dim = 1 << n;
  return (dim / qpd::wg_mtc(n)) * (2 * dim / 256);
}
WgGeom wg_geom(const qp_plan* pl, int64_t nkc) {
  WgGeom g;
  g.tiles = wg_tiles(pl);
  const int64_t T = (int64_t)g.tiles * (nkc > 0 ? nkc : 0);
  g.grid = (int)(T > 0 && T < pl->sm_count ? T : pl->sm_count);
  if (g.grid < g.tiles && T >= g.tiles) g.grid = g.tiles;   // a range then meets at most two tiles
  // n <= 8: a multiple of the tile count, so that every range lies inside one tile (the
  // kernel's second segment is compiled out there); T itself is one
  if (pl->c.n_qubits <= 8) g.grid = g.grid / g.tiles * g.tiles;
  const int64_t per = T > 0 ? (T + g.grid - 1) / g.grid : 1;
  const int64_t flmax = wg_rows_per_chunk(pl) / qpd::WKC;
  const int64_t nfl = (per + flmax - 1) / flmax;
  g.fl = (int)((per + nfl - 1) / nfl);
  g.nslots = 1;
  for (int t = 0; t < g.tiles && T > 0; ++t) {
    const int64_t m = qpd::wg_cta_of((int64_t)(t + 1) * nkc - 1, T, g.grid) - qpd::wg_cta_of((int64_t)t * nkc, T, g.grid) + 1;
    if (m > g.nslots) g.nslots = m;
  }
  return g;
}
// Partial slots the workspace holds: SMs / tiles where the SMs divide evenly over the tiles
// (every range then lies inside one tile), else at most 2 ceil(SMs / tiles) + 2 ranges meet a
// tile.
int64_t wg_slots_cap(const qp_plan* pl) {
  const int t = wg_tiles(pl);
  if (pl->sm_count % t == 0 || pl->c.n_qubits <= 8) return pl->sm_count / t;
  return 2 * ((pl->sm_count + t - 1) / t) + 2;
}

bool dense_path(const qp_plan* pl) { return pl->path == QP_PATH_GEMM_SPLIT; }

int al4(int x);
bool mlp_fused_out(const qp_plan* pl);

// Kernels launched by launch_front: gate preparation, the CRZ mesh diagonal (CRZ ansatze), the
// premap (one kernel, or layer by layer the weight copy, the features and one activation kernel
// per layer, the output layer's own or folded into the last hidden layer's; the layers'
// library GEMMs are not counted).
int front_launches(const qp_plan* pl) {
  const int D = pl->c.mlp_depth;
  return (qp_has_crz(pl->c.ansatz) ? 2 : 1) + (pl->deep ? (mlp_fused_out(pl) ? D + 2 : D + 3) : 1);
}
// Kernels of the premap backward: the fused per-point kernels (1 or 2), or layer by layer the
// output layer (with the last hidden layer's tanh backward and its own weight gradient when
// folded), the bias gradient and the dW slot copy per layer, the tanh backward per hidden layer
// and the period's two kernels with the periodic map.
int premap_bwd_launches(const qp_plan* pl) {
  const int D = pl->c.mlp_depth, per = pl->c.periodic ? 2 : 0;
  if (!pl->deep) return pl->pg_ok ? 1 : 2;
  return mlp_fused_out(pl) ? 1 + 2 * D + (D - 1) + per : 1 + 2 * (D + 1) + D + per;
}

// The fused forward kernel keeps a tile's whole output row (2^(n+1) FP32 columns) in tensor
// memory, which holds 512 columns: n = 7 and 8.
bool fused_path(const qp_plan* pl) {
  return dense_path(pl) && pl->c.n_qubits >= 7 && pl->c.n_qubits <= 8;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// The CUDA driver's tensor-map encoder, through the runtime's entry-point query (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// Tensor maps of the blocked costate buffer [nblk][rtot][256] for the fused forward's bulk
// stores: per point set, its rows (4 per collocation point, 1 per IC/BC point) as (column,
// row, block). Each map's row extent is its set's, so the last, partial tile is clipped.
bool lam_maps(float* lam, int64_t rtot, const int64_t npts[3], int nblk, CUtensorMap m[3]) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
  if (!enc) return false;
  const cuuint32_t es[3] = {1, 1, 1};
  for (int set = 0; set < 3; ++set) {
    const int64_t row0 = set == 0 ? 0 : 4 * npts[0] + (set == 2 ? npts[1] : 0);
    const int64_t rows = set == 0 ? 4 * npts[0] : npts[set];
    const cuuint64_t dims[3] = {256, (cuuint64_t)(rows > 0 ? rows : 1), (cuuint64_t)nblk};
    const cuuint64_t str[2] = {1024, (cuuint64_t)rtot * 1024};
    const cuuint32_t box[3] = {32, 128, 1};
    if (enc(&m[set], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, lam + row0 * 256, dims, str, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// Slot groups of the weight-gradient partial sum: enough blocks to cover the GPU.
int gsum_groups(const qp_plan* pl) {
  const int64_t dd = (int64_t)1 << (2 * pl->c.n_qubits);
  const int64_t g = ((int64_t)pl->sm_count * 8 * 256 + dd - 1) / dd;
  return (int)(g < 1 ? 1 : (g > 8 ? 8 : g));
}

// Layer-by-layer premap: every row buffer has its width rounded up to four floats (al4), so
// that its rows are 16-byte aligned. The layers' weight matrices are copied as
// [al4(out)][al4(in)] to 256-byte aligned offsets (floats from the copy's start; l = depth + 1 gives the total),
// and each weight-gradient chunk writes its dW into a scratch row of the largest layer's size.
int al4(int x) { return (x + 3) & ~3; }
// The output layer folded into the kernels that pass over the last hidden layer's rows (a
// hidden layer exists, at most 128 hidden units, at most 16 angles).
bool mlp_fused_out(const qp_plan* pl) {
  return pl->deep && pl->c.mlp_depth >= 1 && al4(pl->c.mlp_width) <= 128 && pl->c.n_qubits <= 16;
}
int64_t mlp_wcopy_off(const qp_plan* pl, int l) {
  const int F = pl->c.rff_freqs, H = pl->c.mlp_width, D = pl->c.mlp_depth;
  int64_t o = 0;
  int fan = 2 * F;
  for (int i = 0; i < l; ++i) {
    const int out = i == D ? pl->c.n_qubits : H;
    o += ((int64_t)al4(out) * al4(fan) + 63) / 64 * 64;
    fan = H;
  }
  return o;
}
int64_t mlp_dw_stride(const qp_plan* pl) {
  const int F = pl->c.rff_freqs, H = pl->c.mlp_width, D = pl->c.mlp_depth;
  int64_t m = 0;
  int fan = 2 * F;
  for (int i = 0; i <= D; ++i) {
    const int out = i == D ? pl->c.n_qubits : H;
    m = std::max(m, (int64_t)al4(out) * al4(fan));
    fan = H;
  }
  return (m + 63) / 64 * 64;
}

WsLayout ws_layout(const qp_plan* pl, int64_t P0) {
  WsLayout w;
  // with the symmetry penalty the main pass also evaluates up to two mirrored copies of every
  // collocation point
  const bool sym = pl->p.w_sym > 0.f;
  const int64_t P = sym ? 3 * P0 : P0;
  const int n = pl->c.n_qubits, H = pl->c.premap == QP_PREMAP_RFF_MLP ? pl->c.mlp_width : 0;
  size_t o = 0;
  w.status = o; o = al256(o + 256);
  w.gates = o; o = al256(o + (size_t)QP_MAXL * QP_MAXQ * 8 * 4);
  w.cmat = o; o = al256(o + (size_t)QP_MAXL * QP_MAXQ * 3 * 4 * 4);
  w.cenc = o; o = al256(o + (size_t)QP_MAXQ * 4 * 4);
  const bool crz = qp_has_crz(pl->c.ansatz);
  w.crz = o; o = al256(o + (crz ? (size_t)pl->c.n_layers * ((size_t)1 << n) * 8 : 0));
  w.crz64 = o; o = al256(o + (crz && dense_path(pl) ? (size_t)pl->c.n_layers * ((size_t)1 << n) * 16 : 0));
  w.thetaJ = o; o = al256(o + (size_t)P * n * 16);
  w.dthetaJ = o; o = al256(o + (size_t)P * n * 16);
  w.d1 = o; o = al256(o + (size_t)P * H * 16);
  w.d2 = o; o = al256(o + (size_t)(H ? P : 0) * n * 16);
  w.u1 = o; o = al256(o + (size_t)P * H * 16);
  const int nt = pl->p.energy_nt;
  w.blk_loss = o; o = al256(o + (size_t)pl->blocks_grad * (QP_NLP + nt) * 8);
  w.blk_grad = o; o = al256(o + (size_t)pl->blocks_grad * (pl->nE + 3 * pl->c.n_readout + 3) * 4);
  const int64_t nW = H ? pl->mlp_count - pl->nfixed : 0;
  w.wpart = o; o = al256(o + (size_t)pl->nwblk * nW * 4);
  // layer-by-layer premap: (y0, z_x, z_y, z_t) of every hidden layer, and two cotangent
  // buffers of the widest layer
  const int64_t mw = pl->deep ? std::max(al4(H), al4(n)) : 0;
  w.mact = o; o = al256(o + (pl->deep ? (size_t)pl->c.mlp_depth * P * 4 * al4(H) * 4 : 0));
  w.mcot = o; o = al256(o + (size_t)2 * P * 4 * mw * 4);
  w.sxb = o; o = al256(o + (sym ? (size_t)P * 3 * 4 : 0));
  w.sF = o; o = al256(o + (sym ? (size_t)P * 3 * 4 : 0));
  w.sgs = o; o = al256(o + (sym ? (size_t)P0 * 3 * 4 : 0));
  w.sge = o; o = al256(o + (sym ? (size_t)2 * P0 * 3 * 4 : 0));
  w.spart = o; o = al256(o + (sym ? (size_t)pl->sm_count * 4 * 8 : 0));
  w.mtg = o; o = al256(o + (pl->c.periodic ? 8 : 0));
  w.desc = o; o = al256(o + (dense_path(pl) ? 0 : sizeof(QPCircArgs)));
  w.mx0 = o; o = al256(o + (pl->deep ? (size_t)P * 4 * al4(2 * pl->c.rff_freqs) * 4 : 0));
  w.blasws = o; o = al256(o + (pl->deep ? kBlasWorkspace : 0));
  w.mwt = o; o = al256(o + (pl->deep ? (size_t)mlp_wcopy_off(pl, pl->c.mlp_depth + 1) * 4 : 0));
  w.mdw = o; o = al256(o + (pl->deep ? (size_t)pl->nwblk * mlp_dw_stride(pl) * 4 : 0));
  const size_t dim = (size_t)1 << n;
  const bool dn = dense_path(pl);
  w.dW = o; o = al256(o + (dn ? 2 * (2 * dim) * dim * 4 : 0));
  w.dphi = o; o = al256(o + (dn ? (size_t)P * 4 * dim * 8 : 0));
  const bool dg = dn && n >= 7;
  w.dU = o; o = al256(o + (dg ? dim * dim * 16 : 0));
  w.dG = o; o = al256(o + (dg ? dim * dim * 8 : 0));
  w.dY = o; o = al256(o + (dg ? dim * dim * 8 : 0));
  // upper bound of the weight-gradient partial slots: 16-row steps of 4 P rows, plus one per
  // set boundary
  const int64_t nch = dg ? wg_slots_cap(pl) : 0;
  w.dpart = o; o = al256(o + (size_t)nch * dim * 2 * dim * 4);
  const bool dm = dg && pl->c.premap == QP_PREMAP_RFF_MLP;
  w.dWT = o; o = al256(o + (dm ? 2 * (2 * dim) * dim * 4 : 0));
  w.dmu = o; o = al256(o + (dm && !fused_path(pl) ? (size_t)P * 4 * dim * 4 : 0));
  w.dW16 = o; o = al256(o + (dg ? 2 * (2 * dim) * dim * 2 : 0));
  w.dcs = o; o = al256(o + (dg ? (size_t)P * n * 8 : 0));
  w.dgs = o; o = al256(o + (dg ? (size_t)gsum_groups(pl) * dim * dim * 16 : 0));
  w.dgates = o; o = al256(o + (dn ? (size_t)pl->c.n_layers * n * 4 * 16 : 0));
  w.total = o;
  return w;
}

template <int NQ, bool GRAD>
void* circuit_fn(bool crz) {
  return crz ? (void*)qpk::circuit_kernel<NQ, GRAD, true> : (void*)qpk::circuit_kernel<NQ, GRAD, false>;
}

// The statevector kernel of n qubits; crz: the CRZ-mesh form (the other ansatze use the one
// compiled without it).
void* circuit_kernel_ptr(int n, bool grad, bool crz) {
  switch (n) {
#define QP_CASE(N) case N: return grad ? circuit_fn<N, true>(crz) : circuit_fn<N, false>(crz);
    QP_CASE(1) QP_CASE(2) QP_CASE(3) QP_CASE(4) QP_CASE(5)
    QP_CASE(6) QP_CASE(7) QP_CASE(8) QP_CASE(9) QP_CASE(10)
#undef QP_CASE
  }
  return nullptr;
}

void* premap_fwd_ptr(int H) {
  switch (H) {
    case 4: return (void*)qpk::premap_fwd_kernel<4>;
    case 8: return (void*)qpk::premap_fwd_kernel<8>;
    case 16: return (void*)qpk::premap_fwd_kernel<16>;
    case 32: return (void*)qpk::premap_fwd_kernel<32>;
    case 64: return (void*)qpk::premap_fwd_kernel<64>;
  }
  return nullptr;
}
void* premap_fwd4_ptr(int H) {
  switch (H) {
    case 4: return (void*)qpk::premap_fwd4_kernel<4>;
    case 8: return (void*)qpk::premap_fwd4_kernel<8>;
    case 16: return (void*)qpk::premap_fwd4_kernel<16>;
    case 32: return (void*)qpk::premap_fwd4_kernel<32>;
    case 64: return (void*)qpk::premap_fwd4_kernel<64>;
  }
  return nullptr;
}
void* premap_bwd4_ptr(int H) {
  switch (H) {
    case 4: return (void*)qpk::premap_bwd4_kernel<4>;
    case 8: return (void*)qpk::premap_bwd4_kernel<8>;
    case 16: return (void*)qpk::premap_bwd4_kernel<16>;
    case 32: return (void*)qpk::premap_bwd4_kernel<32>;
    case 64: return (void*)qpk::premap_bwd4_kernel<64>;
  }
  return nullptr;
}
void* premap_bwd_ptr(int H) {
  switch (H) {
    case 4: return (void*)qpk::premap_bwd_kernel<4>;
    case 8: return (void*)qpk::premap_bwd_kernel<8>;
    case 16: return (void*)qpk::premap_bwd_kernel<16>;
    case 32: return (void*)qpk::premap_bwd_kernel<32>;
    case 64: return (void*)qpk::premap_bwd_kernel<64>;
  }
  return nullptr;
}

qp_status validate(const qp_circuit* c, const qp_problem* p, int32_t path) {
  if (!c || !p) return QP_ERR_INVALID_ARG;
  if (c->n_qubits < 1 || c->n_qubits > QP_MAXQ) return QP_ERR_INVALID_ARG;
  if (c->n_layers < 1 || c->n_layers > QP_MAXL) return QP_ERR_INVALID_ARG;
  if (c->n_readout < 1 || c->n_readout > c->n_qubits) return QP_ERR_INVALID_ARG;
  if (c->ansatz < 0 || c->ansatz > 6 || c->enc < 0 || c->enc > 1) return QP_ERR_INVALID_ARG;
  if (c->scale < 0 || c->scale > 4) return QP_ERR_INVALID_ARG;
  if (c->premap == QP_PREMAP_DIRECT) {
    if (c->n_direct < 0 || c->n_direct > 3 || c->n_direct > c->n_qubits) return QP_ERR_INVALID_ARG;
  } else if (c->premap == QP_PREMAP_RFF_MLP) {
    if (c->rff_freqs < 1 || c->mlp_width < 1 || c->mlp_depth < 0) return QP_ERR_INVALID_ARG;
    if (c->periodic != 0 && c->periodic != 1) return QP_ERR_INVALID_ARG;
    // any depth and width up to these bounds (the layer-by-layer kernels)
    if (c->rff_freqs > QP_MAXF || c->mlp_width > 1024 || c->mlp_depth > 8) return QP_ERR_UNSUPPORTED;
  } else {
    return QP_ERR_INVALID_ARG;
  }
  if (c->premap != QP_PREMAP_RFF_MLP && c->periodic != 0) return QP_ERR_INVALID_ARG;
  if (p->medium != QP_MEDIUM_VACUUM && p->medium != QP_MEDIUM_DIELECTRIC) return QP_ERR_INVALID_ARG;
  if (p->phys_loss < 0 || p->phys_loss > 1 || !(p->w_sym >= 0.f)) return QP_ERR_INVALID_ARG;
  if (p->energy_nt < 0 || p->energy_nt > QP_MAXNT || p->energy_slice < 0) return QP_ERR_INVALID_ARG;
  if (p->medium == QP_MEDIUM_DIELECTRIC && !(p->sigmoid_w > 0.f)) return QP_ERR_INVALID_ARG;
  if (!(p->ic_sigma > 0.f)) return QP_ERR_INVALID_ARG;
  if (path == QP_PATH_GEMM_SPLIT) {
    if (c->n_qubits < 5) return QP_ERR_UNSUPPORTED;  // K = 2^n must hold one 32-wide chunk
  } else if (path != QP_PATH_AUTO && path != QP_PATH_SIMT_FP32) {
    return QP_ERR_UNSUPPORTED;
  }
  return QP_OK;
}

qp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? QP_OK : QP_ERR_CUDA; }

}  // namespace

extern "C" {

const char* qp_status_str(qp_status s) {
  switch (s) {
    case QP_OK: return "ok";
    case QP_ERR_INVALID_ARG: return "invalid argument";
    case QP_ERR_UNSUPPORTED: return "unsupported configuration";
    case QP_ERR_BUFFER_TOO_SMALL: return "workspace missing or too small";
    case QP_ERR_CUDA: return "CUDA error";
    case QP_ERR_NONFINITE: return "non-finite loss";
    case QP_ERR_TIMEOUT: return "device wait timed out";
    case QP_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

qp_status qp_plan_create(const qp_circuit* circuit, const qp_problem* problem, int32_t path,
                         qp_plan** out) {
  if (!out) return QP_ERR_INVALID_ARG;
  *out = nullptr;
  qp_status st = validate(circuit, problem, path);
  if (st != QP_OK) return st;
  qp_plan* pl = new (std::nothrow) qp_plan();
  if (!pl) return QP_ERR_INTERNAL;
  pl->c = *circuit;
  pl->p = *problem;
  // AUTO: the fused-unitary tensor-core path where it is faster and stays within 1e-5 of the
  // FP64 reference (7-10 qubits: at 7 qubits 2x the gate-by-gate speed at 2 layers, 4.5x at 6);
  // the FP32 gate-by-gate path otherwise.
  pl->path = path != QP_PATH_AUTO ? path
             : (circuit->n_qubits >= 7 ? QP_PATH_GEMM_SPLIT : QP_PATH_SIMT_FP32);
  const int n = circuit->n_qubits;
  if (qp_build_sched(n, circuit->n_layers, circuit->ansatz, &pl->sched) != 0) {
    delete pl;
    return QP_ERR_UNSUPPORTED;
  }
  pl->mlp_count = premap_count(*circuit);
  pl->nfixed = omega_count(*circuit);
  pl->mlp_off = pl->nfixed;
  pl->circ_off = pl->mlp_count;
  pl->head_off = pl->circ_off + (int64_t)circuit->n_layers * qp_layer_params(circuit->ansatz, n);
  pl->nE = 3 * n * circuit->n_layers + circuit->n_layers * qp_crz_sums(circuit->ansatz, n);
  pl->n_params = pl->head_off + 3LL * circuit->n_readout + 3;

  if (cudaGetDevice(&pl->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device) != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return QP_ERR_CUDA;
  }
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
  const int dim = 1 << n, ppw = geo_ppw(n);
  const int nt = problem->energy_nt;
  for (int g = 0; g < 2; ++g) {
    const bool grad = g == 0;
    const int nvec = grad ? 8 : 4;
    const int sstride = nvec * dim + (n <= 3 ? 1 : 0);
    int warps = kMaxWarps;
    qpk::SmemLayout lay;
    for (; warps >= 1; --warps) {
      lay = qpk::smem_layout(n, circuit->n_layers, circuit->n_readout, grad ? nt : 0, warps, sstride, ppw, pl->nE);
      if (lay.total <= smem_optin) break;
    }
    if (warps < 1) { delete pl; return QP_ERR_UNSUPPORTED; }
    void* fn = circuit_kernel_ptr(n, grad, qp_has_crz(circuit->ansatz));
    if (raise_smem_limit(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lay.total) != cudaSuccess) {
      cudaGetLastError();
      delete pl;
      return QP_ERR_CUDA;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, lay.total);
    if (per_sm < 1) per_sm = 1;
    if (grad) {
      pl->warps_grad = warps; pl->smem_grad = lay.total; pl->sstride_grad = sstride;
      pl->blocks_grad = pl->sm_count * per_sm;
    } else {
      pl->warps_fwd = warps; pl->smem_fwd = lay.total; pl->sstride_fwd = sstride;
      pl->blocks_fwd = pl->sm_count * per_sm;
    }
  }
  if (dense_path(pl)) {
    if (cudaStreamCreateWithFlags(&pl->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      delete pl;
      return QP_ERR_CUDA;
    }
    if (raise_smem_limit((void*)qpd::dense_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * (1 << n) * 16) != cudaSuccess ||
        raise_smem_limit((void*)qpd::dense_row_gemm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             qpd::gemm_smem_bytes(n, 0)) != cudaSuccess ||
        raise_smem_limit((void*)qpd::dense_row_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             qpd::gemm_smem_bytes(n, 1)) != cudaSuccess ||
        raise_smem_limit((void*)qpd::dense_row16_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         qpd::row16_smem_bytes()) != cudaSuccess ||
        raise_smem_limit((void*)qpd::dense_row16_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         qpd::row16_smem_bytes()) != cudaSuccess ||
        raise_smem_limit(wgrad_kernel<false>(n), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             qpd::wgc_smem(n, false).total) != cudaSuccess ||
        raise_smem_limit(wgrad_kernel<true>(n), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             qpd::wgc_smem(n, true).total) != cudaSuccess ||
        raise_smem_limit((void*)qpd::dense_sweep_left_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (1 << n) * 16 * 8) != cudaSuccess ||
        raise_smem_limit((void*)qpd::dense_sweep_right_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (1 << n) * 16 * 8) != cudaSuccess ||
        (n <= 8 && raise_smem_limit((void*)qpd::dense_sweep_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    qpd::swc_smem(n, pl->c.n_layers, qpd::swc_size(n, false), qp_crz_sums(pl->c.ansatz, n))) != cudaSuccess) ||
        (fused_path(pl) &&
         (raise_smem_limit(n == 7 ? (void*)qpd::dense_fused_fwd_kernel<7> : (void*)qpd::dense_fused_fwd_kernel<8>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           qpd::fused_smem(n, pl->p.energy_nt).total) != cudaSuccess ||
          raise_smem_limit(n == 7 ? (void*)qpd::dense_mu_embed_kernel<7> : (void*)qpd::dense_mu_embed_kernel<8>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, qpd::mu_smem_bytes(n)) != cudaSuccess))) {
      cudaGetLastError();
      delete pl;
      return QP_ERR_CUDA;
    }
    if (n >= 4 && n <= 8) {
      // a 16-CTA cluster (non-portable size) halves every CTA's share of the sweep
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(qpd::SWC_THREADS);
      cfg.dynamicSmemBytes = qpd::swc_smem(n, pl->c.n_layers, 16, qp_crz_sums(pl->c.ansatz, n));
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      pl->swc_big = cudaFuncSetAttribute((const void*)qpd::dense_sweep_cluster_kernel,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
                    cudaOccupancyMaxActiveClusters(&nclusters, (const void*)qpd::dense_sweep_cluster_kernel, &cfg) ==
                        cudaSuccess &&
                    nclusters >= 1;
      cudaGetLastError();
    }
  }
  if (circuit->premap == QP_PREMAP_RFF_MLP) {
    const int F = circuit->rff_freqs, H = circuit->mlp_width;
    pl->smem_premap = (H * 2 * F + H + n * H + n + 3 * F) * 4;
    pl->nwblk = pl->sm_count * 2;
    int tile = 32;
    while (tile > 1 && (tile * (2 * F + 2 * H + n) * 16 + 3 * F * 4) > 96 * 1024) tile >>= 1;
    pl->wtile = tile;
    pl->smem_wgrad = tile * (2 * F + 2 * H + n) * 16 + 3 * F * 4;
    pl->smem_premap4 = qpk::premap4_smem(F, H, n);
    // one hidden layer of a width the fused per-point kernels take; otherwise layer by layer
    const bool one_layer = circuit->mlp_depth == 1 && (H == 4 || H == 8 || H == 16 || H == 32 || H == 64) &&
                           (F % 2) == 0 && (int64_t)H * 2 * F <= 16 * 4 * 256 && n * H <= 4 * 256;
    pl->deep = !one_layer || circuit->periodic;
    // FP32 GEMMs emulated on the tensor cores (BF16x9: FP32 accuracy) wherever the library has
    // them, without the special-value scans (the weight copy flags non-finite weights)
    static_assert(qpm::MLP_MAX_LAYERS >= 9, "depth 8 premaps have nine layers");
    if (pl->deep && (cublasCreate(&pl->blas) != CUBLAS_STATUS_SUCCESS ||
                     cublasSetEmulationStrategy(pl->blas, CUBLAS_EMULATION_STRATEGY_EAGER) != CUBLAS_STATUS_SUCCESS ||
                     cublasSetEmulationSpecialValuesSupport(pl->blas, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE) !=
                         CUBLAS_STATUS_SUCCESS)) {
      delete pl;
      return QP_ERR_CUDA;
    }
    pl->pg_ok = one_layer && F == qpk::PG_F && H == qpk::PG_H && n <= 16;
    if (pl->pg_ok &&
        (raise_smem_limit((void*)qpk::premap_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          qpk::pt_smem(n).total) != cudaSuccess ||
         raise_smem_limit((void*)qpk::premap_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          qpk::pb_smem(n)) != cudaSuccess)) {
      cudaGetLastError();
      delete pl;
      return QP_ERR_CUDA;
    }
    if (!pl->deep &&
        (raise_smem_limit(premap_fwd_ptr(H), cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem_premap) != cudaSuccess ||
        raise_smem_limit(premap_fwd4_ptr(H), cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem_premap4) != cudaSuccess ||
        raise_smem_limit(premap_bwd4_ptr(H), cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem_premap4) != cudaSuccess ||
        raise_smem_limit(premap_bwd_ptr(H), cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem_premap) != cudaSuccess ||
        raise_smem_limit((void*)qpk::premap_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->smem_wgrad) != cudaSuccess)) {
      cudaGetLastError();
      delete pl;
      return QP_ERR_CUDA;
    }
  }
  *out = pl;
  return QP_OK;
}

void qp_plan_destroy(qp_plan* plan) { delete plan; }

qp_status qp_param_count(const qp_plan* plan, int64_t* n_params) {
  if (!plan || !n_params) return QP_ERR_INVALID_ARG;
  *n_params = plan->n_params;
  return QP_OK;
}

qp_status qp_param_layout(const qp_plan* plan, int64_t* o) {
  if (!plan || !o) return QP_ERR_INVALID_ARG;
  o[0] = plan->circ_off; o[1] = plan->head_off; o[2] = plan->n_params; o[3] = plan->nfixed;
  return QP_OK;
}

qp_status qp_workspace_size(const qp_plan* plan, int64_t max_points, size_t* bytes) {
  if (!plan || !bytes || max_points < 0) return QP_ERR_INVALID_ARG;
  *bytes = ws_layout(plan, max_points).total;
  return QP_OK;
}

qp_status qp_set_workspace(qp_plan* plan, void* d_ws, size_t bytes) {
  if (!plan || (bytes && !d_ws)) return QP_ERR_INVALID_ARG;
  if (((uintptr_t)d_ws & 255) != 0) return QP_ERR_INVALID_ARG;
  // the status word lives at the start of the workspace: follow it to the new one
  if (plan->ws && plan->last_status == (const int32_t*)plan->ws) plan->last_status = (const int32_t*)d_ws;
  plan->ws = d_ws;
  plan->ws_bytes = bytes;
  return QP_OK;
}

int32_t qp_last_launch_count(const qp_plan* plan) { return plan ? plan->last_launches : -1; }

int32_t qp_plan_path(const qp_plan* plan) { return plan ? plan->path : -1; }

qp_status qp_bh_indicator(const double* d_loss_terms, int32_t energy_nt, double t_max, double delta,
                          double* d_out, void* stream) {
  if (!d_loss_terms || !d_out || energy_nt < 2 || energy_nt > QP_MAXNT || !(t_max > 0.0) ||
      !(delta >= 0.0 && delta <= t_max))
    return QP_ERR_INVALID_ARG;
  // first slice with t_k >= delta (the same relative slack as the FP64 reference)
  const double kf = std::ceil((delta / t_max - 1e-12) * (energy_nt - 1));
  const int k0 = kf < 0.0 ? 0 : (kf > energy_nt - 1 ? energy_nt - 1 : (int)kf);
  qpk::bh_indicator_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(d_loss_terms + QP_NLOSS, energy_nt, k0, d_out);
  return cuda_status(cudaGetLastError());
}

qp_status qp_plan_set_operands(qp_plan* plan, int32_t operands) {
  if (!plan || (operands != QP_OPERANDS_FP16_PAIRS && operands != QP_OPERANDS_TF32_PAIRS))
    return QP_ERR_INVALID_ARG;
  plan->operands = operands;
  return QP_OK;
}

qp_status qp_set_wait_limit(qp_plan* plan, uint32_t polls) {
  if (!plan) return QP_ERR_INVALID_ARG;
  plan->wait_limit = polls;
  return QP_OK;
}

qp_status qp_set_profile_events(qp_plan* plan, int32_t kernel, void* ev_start, void* ev_stop) {
  if (!plan || kernel < 0 || kernel > 2 || ((ev_start == nullptr) != (ev_stop == nullptr)))
    return QP_ERR_INVALID_ARG;
  plan->prof_start[kernel] = (cudaEvent_t)ev_start;
  plan->prof_stop[kernel] = (cudaEvent_t)ev_stop;
  return QP_OK;
}

// Record the plan's profiling event of `kernel` (start or stop), if it has one.
static void prof_mark(const qp_plan* pl, int kernel, bool start, cudaStream_t s) {
  const cudaEvent_t e = start ? pl->prof_start[kernel] : pl->prof_stop[kernel];
  if (e) cudaEventRecord(e, s);
}

static void fill_problem(const qp_plan* pl, QPProblemDev& d) {
  const qp_problem& p = pl->p;
  d.medium = p.medium; d.eps_r = p.eps_r; d.disk_r = p.disk_r; d.disk_x0 = p.disk_x0;
  d.disk_y0 = p.disk_y0; d.sigmoid_w = p.sigmoid_w; d.ic_sigma = p.ic_sigma; d.ic_x0 = p.ic_x0;
  d.ic_y0 = p.ic_y0; d.w_ic = p.w_ic; d.w_bc = p.w_bc; d.w_energy = p.w_energy;
  d.energy_slice = p.energy_slice; d.energy_nt = p.energy_nt;
  d.phys_loss = p.phys_loss; d.w_sym = p.w_sym;
  for (int i = 0; i < 3; ++i) d.norm[i] = pl->cur_norm[i];
  d.norm_diel = pl->cur_norm_diel;
  d.colloc_off = pl->cur_colloc_off;
}

// MLP layer l of the layer-by-layer premap (0 .. depth - 1 hidden, depth the output layer):
// input and output widths, offsets of its W [out][in] and b [out] after the Omega entries.
static void mlp_layer_geom(const qp_plan* pl, int l, int& in, int& out, int64_t& w_off, int64_t& b_off) {
  const int F = pl->c.rff_freqs, H = pl->c.mlp_width, D = pl->c.mlp_depth;
  int64_t o = pl->c.periodic ? 1 : 0;   // the learned period comes first
  int fan = 2 * F;
  for (int i = 0; i < l; ++i) { o += (int64_t)H * fan + H; fan = H; }
  in = fan;
  out = l == D ? pl->c.n_qubits : H;
  w_off = o;
  b_off = o + (int64_t)out * in;
}

static qpm::MlpArgs mlp_layer_args(const qp_plan* pl, const float* d_params, const float* const pts[3],
                                   const int64_t npts[3], const WsLayout& w, int l) {
  char* ws = (char*)pl->ws;
  qpm::MlpArgs m;
  std::memset(&m, 0, sizeof(m));
  m.n4 = npts[0] + npts[1] + npts[2];   // four rows for every point unless a caller says otherwise
  for (int i = 0; i < 3; ++i) { m.pts[i] = pts[i]; m.npts[i] = npts[i]; }
  m.ptot = npts[0] + npts[1] + npts[2];
  m.omega = d_params;
  m.F = pl->c.rff_freqs;
  m.period = pl->c.periodic ? d_params + pl->nfixed : nullptr;
  int64_t wo, bo;
  mlp_layer_geom(pl, l, m.in, m.out, wo, bo);
  m.W = d_params + pl->nfixed + wo;
  m.b = d_params + pl->nfixed + bo;
  m.ldi = al4(m.in);
  m.ldo = al4(m.out);
  const int64_t lstride = m.ptot * 4 * al4(pl->c.mlp_width);
  m.act_in = l > 0 ? (const float*)(ws + w.mact) + (int64_t)(l - 1) * lstride : nullptr;
  m.act_out = l == pl->c.mlp_depth ? nullptr : (float*)(ws + w.mact) + (int64_t)l * lstride;
  m.scale = pl->c.scale;
  m.thetaJ = (float*)(ws + w.thetaJ);
  m.hout = (float*)(ws + w.d2);
  m.counts = (int32_t*)(ws + w.status) + 1;
  m.medium = pl->p.medium;
  m.disk_r = pl->p.disk_r; m.disk_x0 = pl->p.disk_x0; m.disk_y0 = pl->p.disk_y0;
  return m;
}

static int mlp_grid(const qp_plan* pl, int64_t tiles) {
  const int64_t cap = (int64_t)pl->sm_count * 4;
  return (int)(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
}

// Library GEMM of the layer-by-layer premap on the plan's handle, column-major arguments
// (C = op(A) op(B), alpha 1). The first call that the emulated FP32 compute type does not
// accept switches the plan to plain FP32. A GEMM with a dimension below 32 besides the rows
// (the output layer's few angles) runs in plain FP32: the emulated kernels' tiles would be
// mostly padding.
static qp_status mlp_gemm(qp_plan* pl, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k,
                          const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                          long long sa = 0, long long sb = 0, long long sc = 0, int batch = 0) {
  const float one = 1.f, zero = 0.f;
  const int narrow = std::min(std::min(m, n), k);   // the row count is the largest of the three
  for (;;) {
    const cublasComputeType_t ct = narrow < 32 ? CUBLAS_COMPUTE_32F : pl->blas_ct;
    const cublasStatus_t st = batch > 0
        ? cublasGemmStridedBatchedEx(pl->blas, ta, tb, m, n, k, &one, A, CUDA_R_32F, lda, sa, B, CUDA_R_32F, ldb,
                                     sb, &zero, C, CUDA_R_32F, ldc, sc, batch, ct, CUBLAS_GEMM_DEFAULT)
        : cublasGemmEx(pl->blas, ta, tb, m, n, k, &one, A, CUDA_R_32F, lda, B, CUDA_R_32F, ldb, &zero, C,
                       CUDA_R_32F, ldc, ct, CUBLAS_GEMM_DEFAULT);
    if (st == CUBLAS_STATUS_SUCCESS) return QP_OK;
    if (ct == CUBLAS_COMPUTE_32F ||
        (st != CUBLAS_STATUS_NOT_SUPPORTED && st != CUBLAS_STATUS_INVALID_VALUE))
      return QP_ERR_CUDA;
    pl->blas_ct = CUBLAS_COMPUTE_32F;
  }
}

// Binds the plan's handle to the call's stream and workspace (no allocation, so the calls
// can be captured into a graph).
static qp_status mlp_blas_bind(qp_plan* pl, const WsLayout& w, cudaStream_t s) {
  if (cublasSetStream(pl->blas, s) != CUBLAS_STATUS_SUCCESS ||
      cublasSetWorkspace(pl->blas, (char*)pl->ws + w.blasws, kBlasWorkspace) != CUBLAS_STATUS_SUCCESS)
    return QP_ERR_CUDA;
  return QP_OK;
}

static int ew_grid(const qp_plan* pl, int64_t n) {
  const int64_t b = (n + 255) / 256, cap = (int64_t)pl->sm_count * 8;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

// Forward of the layer-by-layer premap: the RFF features of every point, then per layer the
// contraction of all (point, s) rows as one library GEMM and its activation; the output layer
// writes the angles and their Jacobian (and counts the dielectric set).
// n4: the first n4 points carry four rows (values and input tangents), the others one (no
// later stage reads their input derivatives), so the layers' contractions run on 3 n4 + P rows
static qp_status launch_mlp_fwd(qp_plan* pl, const float* d_params, const float* const pts[3],
                                const int64_t npts[3], const WsLayout& w, cudaStream_t s, int64_t n4) {
  char* ws = (char*)pl->ws;
  const int64_t P = npts[0] + npts[1] + npts[2];
  const int D = pl->c.mlp_depth;
  if (4 * P > (int64_t)INT32_MAX) return QP_ERR_UNSUPPORTED;
  const int R = (int)(3 * n4 + P);
  qp_status st = mlp_blas_bind(pl, w, s);
  if (st != QP_OK) return st;
  float* X0 = (float*)(ws + w.mx0);
  float* Wc = (float*)(ws + w.mwt);
  {
    // the layers' weights at aligned offsets (the library's vectorised kernels need them)
    qpm::MlpCopyArgs ca;
    std::memset(&ca, 0, sizeof(ca));
    ca.src = d_params + pl->nfixed;
    ca.dst = Wc;
    ca.nl = D + 1;
    ca.status = (int32_t*)(ws + w.status);
    int64_t most = 0;
    for (int l = 0; l <= D; ++l) {
      int64_t bo;
      mlp_layer_geom(pl, l, ca.in[l], ca.out[l], ca.src_off[l], bo);
      ca.ld[l] = al4(ca.in[l]);
      ca.outp[l] = al4(ca.out[l]);
      ca.dst_off[l] = mlp_wcopy_off(pl, l);
      most = std::max(most, (int64_t)ca.outp[l] * ca.ld[l]);
    }
    qpm::mlp_wcopy_kernel<<<ew_grid(pl, most), 256, 0, s>>>(ca);
  }
  {
    qpm::MlpArgs m0 = mlp_layer_args(pl, d_params, pts, npts, w, 0);
    m0.n4 = n4;
    qpm::mlp_features_kernel<<<ew_grid(pl, P * 32), 256, (size_t)m0.F * (m0.period ? 6 : 3) * 4, s>>>(
        m0, X0, m0.ldi);   // pads zeroed
  }
  const bool fo = mlp_fused_out(pl);
  for (int l = 0; l <= (fo ? D - 1 : D); ++l) {
    qpm::MlpArgs m = mlp_layer_args(pl, d_params, pts, npts, w, l);
    m.n4 = n4;
    const float* X = l == 0 ? X0 : m.act_in;
    float* Hl = l == D ? (float*)(ws + w.mcot) : m.act_out;
    // H[R][out] = X[R][in] W^T: column-major H^T = W X^T (padded sizes: the pads are zero)
    if (R > 0)
      st = mlp_gemm(pl, CUBLAS_OP_T, CUBLAS_OP_N, m.ldo, R, m.ldi, Wc + mlp_wcopy_off(pl, l), m.ldi, X, m.ldi, Hl,
                    m.ldo);
    if (st != QP_OK) return st;
    if (fo && l == D - 1) {
      // the last hidden layer's activation with the output layer, per point
      qpm::MlpArgs mo = mlp_layer_args(pl, d_params, pts, npts, w, D);
      mo.n4 = n4;
      const size_t sm = (size_t)mo.out * mo.ldi * 4;
      if (mo.out <= 8)
        qpm::mlp_act_out_kernel<8><<<ew_grid(pl, P * 32), 256, sm, s>>>(mo, Hl, m.b);
      else
        qpm::mlp_act_out_kernel<16><<<ew_grid(pl, P * 32), 256, sm, s>>>(mo, Hl, m.b);
    } else if (l < D) {
      qpm::mlp_act_kernel<<<ew_grid(pl, P * (m.ldo / 4)), 256, 0, s>>>(Hl, m.b, P, m.out, m.ldo, n4);
    } else {
      qpm::mlp_out_kernel<<<ew_grid(pl, P * m.out), 256, 0, s>>>(Hl, m);
    }
  }
  return cuda_status(cudaGetLastError());
}

// Weight and bias gradients of layer l from its input rows X [R][in] and the cotangents of
// its pre-activations cot [R][out], one partial slot per point chunk (the slots are summed in
// FP64 with the others): dW = cot^T X per chunk as one strided batched GEMM into aligned
// scratch rows, the last partial chunk as one more GEMM, then copied into the slots (the unused
// ones zeroed).
static qp_status mlp_layer_dw(qp_plan* pl, const float* X, const float* cot, int64_t P, int64_t n4, int in, int out,
                              int ldi, int ldo, int64_t w_off, int64_t b_off, const WsLayout& w, cudaStream_t s) {
  float* part = (float*)((char*)pl->ws + w.wpart);
  float* dw = (float*)((char*)pl->ws + w.mdw);
  const int64_t dws = mlp_dw_stride(pl);
  const int64_t nW = pl->mlp_count - pl->nfixed;
  const int nc = pl->nwblk;
  const int64_t chunk = P > nc ? (P + nc - 1) / nc : 1;   // points per slot (bias sums)
  // dW sums over rows, whichever point they belong to: chunks of rc rows
  const int64_t Rr = 3 * n4 + P;
  const int rc = (int)(Rr > nc ? (Rr + nc - 1) / nc : 1);
  const int64_t nfull = Rr / rc, rest = Rr - nfull * rc;
  const int used = (int)(nfull + (rest > 0 ? 1 : 0));
  qp_status st = QP_OK;
  // column-major dW^T [in x out] = X_c^T (in x rc) . cot_c (rc x out), on the padded sizes
  if (nfull > 0)
    st = mlp_gemm(pl, CUBLAS_OP_N, CUBLAS_OP_T, ldi, ldo, rc, X, ldi, cot, ldo, dw, ldi,
                  (long long)rc * ldi, (long long)rc * ldo, (long long)dws, (int)nfull);
  if (st == QP_OK && rest > 0)
    st = mlp_gemm(pl, CUBLAS_OP_N, CUBLAS_OP_T, ldi, ldo, (int)rest, X + nfull * rc * (int64_t)ldi, ldi,
                  cot + nfull * rc * (int64_t)ldo, ldo, dw + nfull * dws, ldi);
  if (st != QP_OK) return st;
  qpm::mlp_db_kernel<<<nc, qpm::DB_THREADS, 0, s>>>(cot, P, out, ldo, chunk, part, nW, b_off, n4);
  qpm::mlp_dw_slots_kernel<<<ew_grid(pl, (int64_t)nc * out * in), 256, 0, s>>>(dw, dws, ldi, part, nW, w_off, in,
                                                                               out, used, nc);
  return QP_OK;
}

// Backward of the layer-by-layer premap from dL/dtheta, dL/dJ: the output layer's cotangents,
// then per layer (last to first) its weight-gradient partials and the cotangents of the
// previous layer (dU = cot W as one library GEMM, then back through that layer's tanh). With
// the periodic map the first layer's input cotangents give the learned period's gradient.
static qp_status launch_mlp_bwd(qp_plan* pl, const float* d_params, const float* const pts[3],
                                const int64_t npts[3], const WsLayout& w, cudaStream_t s) {
  char* ws = (char*)pl->ws;
  const int64_t P = npts[0] + npts[1] + npts[2];
  const int n = pl->c.n_qubits, D = pl->c.mlp_depth, H = pl->c.mlp_width;
  const int64_t mw = std::max(al4(H), al4(n));
  const int64_t nW = pl->mlp_count - pl->nfixed;
  if (4 * P > (int64_t)INT32_MAX) return QP_ERR_UNSUPPORTED;
  // the forward's layout: four rows for the collocation points, one for the others
  const int64_t n4 = npts[0];
  const int R = (int)(3 * n4 + P);
  qp_status st = mlp_blas_bind(pl, w, s);
  if (st != QP_OK) return st;
  float* cot[2] = {(float*)(ws + w.mcot), (float*)(ws + w.mcot) + P * 4 * mw};
  int cur = 0;
  const bool fo = mlp_fused_out(pl);
  if (fo) {
    // output layer, its weight gradient and the last hidden layer's tanh backward, per point
    qpm::MlpArgs mo = mlp_layer_args(pl, d_params, pts, npts, w, D);
    mo.n4 = n4;
    int in, out;
    int64_t w_off, b_off;
    mlp_layer_geom(pl, D, in, out, w_off, b_off);
    const int nc = pl->nwblk;
    const int64_t chunk = P > nc ? (P + nc - 1) / nc : 1;
    const size_t sm = (size_t)(2 * mo.out * mo.ldi + mo.out) * 4;
    if (mo.out <= 8)
      qpm::mlp_out_bwd_kernel<8><<<nc, 256, sm, s>>>(mo, (const float*)(ws + w.d2), (const float*)(ws + w.dthetaJ),
                                                     mo.act_in, cot[cur], chunk, (float*)(ws + w.wpart), nW, w_off,
                                                     b_off);
    else
      qpm::mlp_out_bwd_kernel<16><<<nc, 256, sm, s>>>(mo, (const float*)(ws + w.d2), (const float*)(ws + w.dthetaJ),
                                                      mo.act_in, cot[cur], chunk, (float*)(ws + w.wpart), nW, w_off,
                                                      b_off);
  } else {
    qpm::mlp_bwd_out_kernel<<<ew_grid(pl, P * al4(n)), 256, 0, s>>>((const float*)(ws + w.d2),
                                                               (const float*)(ws + w.dthetaJ), P, n, al4(n),
                                                               pl->c.scale, cot[cur], n4);
  }
  float* X0 = (float*)(ws + w.mx0);
  const float* Wc = (const float*)(ws + w.mwt);   // the forward's aligned weight copies
  for (int l = fo ? D - 1 : D; l >= 0; --l) {
    qpm::MlpArgs m = mlp_layer_args(pl, d_params, pts, npts, w, l);
    m.n4 = n4;
    int in, out;
    int64_t w_off, b_off;
    mlp_layer_geom(pl, l, in, out, w_off, b_off);
    const float* X = l == 0 ? X0 : m.act_in;
    st = mlp_layer_dw(pl, X, cot[cur], P, n4, in, out, m.ldi, m.ldo, w_off, b_off, w, s);
    if (st != QP_OK) return st;
    if (l > 0 || pl->c.periodic) {
      // dU[R][in] = cot[R][out] W: column-major dU^T = W^T cot^T; for the first layer (periodic
      // map) the features' cotangents, over the features, which are no longer needed
      float* dU = l > 0 ? cot[cur ^ 1] : X0;
      if (R > 0)
        st = mlp_gemm(pl, CUBLAS_OP_N, CUBLAS_OP_N, m.ldi, R, m.ldo, Wc + mlp_wcopy_off(pl, l), m.ldi, cot[cur],
                      m.ldo, dU, m.ldi);
      if (st != QP_OK) return st;
      if (l > 0) {
        qpm::mlp_dact_kernel<<<ew_grid(pl, P * (m.ldi / 4)), 256, 0, s>>>(dU, m.act_in, P, m.ldi, n4);
        cur ^= 1;
        continue;
      }
      if (cudaMemsetAsync(ws + w.mtg, 0, sizeof(double), s) != cudaSuccess) return QP_ERR_CUDA;
      qpm::mlp_period_kernel<<<ew_grid(pl, P * 32), 256, (size_t)m.F * 6 * 4, s>>>(X0, m, m.ldi,
                                                                                 (double*)(ws + w.mtg));
      qpm::mlp_period_fin_kernel<<<(pl->nwblk + 255) / 256, 256, 0, s>>>(
          (const double*)(ws + w.mtg), (float*)(ws + w.wpart), nW, 0, pl->nwblk);
    }
  }
  return cuda_status(cudaGetLastError());
}

// The tensor-core premap forward also writes the half-angle factors (cos, sin) of theta / 2
// that the tensor-core path's contractions read (otherwise a kernel of their own does).
static bool front_writes_cs(const qp_plan* pl) {
  return dense_path(pl) && pl->c.n_qubits >= 7 && pl->c.premap == QP_PREMAP_RFF_MLP && !pl->deep && pl->pg_ok;
}

// Shared prologue: gate preparation and premap forward for all point sets.
// values_only: the caller reads no input derivatives (the layer-by-layer premap then carries one
// row per point instead of four).
static qp_status launch_front(qp_plan* pl, const float* d_params, const float* const pts[3],
                              const int64_t npts[3], const WsLayout& w, cudaStream_t s, bool grad,
                              bool values_only = false) {
  char* ws = (char*)pl->ws;
  const int n = pl->c.n_qubits, L = pl->c.n_layers;
  qpk::PrepArgs pa;
  pa.params = d_params; pa.circ_off = pl->circ_off; pa.n = n; pa.L = L;
  pa.ansatz = pl->c.ansatz; pa.enc = pl->c.enc;
  pa.gates = (float*)(ws + w.gates); pa.cmat = (float*)(ws + w.cmat); pa.cenc = (float*)(ws + w.cenc);
  pa.counts = (int32_t*)(ws + w.status) + 1; pa.status = (int32_t*)(ws + w.status);
  qpk::prep_kernel<<<(L * n + 63) / 64, 64, 0, s>>>(pa);
  if (qp_has_crz(pl->c.ansatz)) {
    // diagonal of every layer's CRZ mesh (FP64 as well for the unitary build)
    const int64_t tot = (int64_t)L << n;
    qpk::crz_phase_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        d_params, pl->circ_off, n, L, pl->c.ansatz, (float2*)(ws + w.crz),
        dense_path(pl) ? (double2*)(ws + w.crz64) : nullptr);
  }
  qpk::PremapArgs ma;
  std::memset(&ma, 0, sizeof(ma));
  for (int i = 0; i < 3; ++i) { ma.pts[i] = pts[i]; ma.npts[i] = npts[i]; }
  ma.ptot = npts[0] + npts[1] + npts[2];
  ma.params = d_params; ma.n = n; ma.premap = pl->c.premap; ma.scale = pl->c.scale;
  ma.n_direct = pl->c.n_direct; ma.F = pl->c.rff_freqs; ma.H = pl->c.mlp_width;
  ma.thetaJ = (float*)(ws + w.thetaJ);
  ma.counts = pa.counts; ma.medium = pl->p.medium; ma.status = pa.status;
  ma.disk_r = pl->p.disk_r; ma.disk_x0 = pl->p.disk_x0; ma.disk_y0 = pl->p.disk_y0;
  const int pblocks = (int)((ma.ptot + 127) / 128 < pl->sm_count * 8 ? (ma.ptot + 127) / 128 : pl->sm_count * 8);
  if (pl->c.premap == QP_PREMAP_RFF_MLP && pl->deep) {
    return launch_mlp_fwd(pl, d_params, pts, npts, w, s, values_only && !grad ? 0 : npts[0]);
  } else if (pl->c.premap == QP_PREMAP_RFF_MLP && pl->pg_ok) {
    // one tensor-core contraction per 128-point tile; the unit table is kept for the backward
    ma.u1 = grad ? (float*)(ws + w.u1) : nullptr;
    if (front_writes_cs(pl)) ma.cs = (float2*)(ws + w.dcs);
    const int64_t nt = (ma.ptot + qpk::PT_M - 1) / qpk::PT_M;   // two CTAs per SM
    const int gb = (int)(nt < 2 * pl->sm_count ? (nt > 0 ? nt : 1) : 2 * pl->sm_count);
    qpk::premap_fwd_tc_kernel<<<gb, qpk::PT_THREADS, qpk::pt_smem(n).total, s>>>(ma);
  } else if (pl->c.premap == QP_PREMAP_RFF_MLP) {
    // four threads per point, 32 points per block
    const int64_t qb = (ma.ptot + 31) / 32;
    const int qblocks = (int)(qb < pl->sm_count * 8 ? (qb > 0 ? qb : 1) : pl->sm_count * 8);
    void* fn = premap_fwd4_ptr(pl->c.mlp_width);
    void* args[] = {&ma};
    if (cudaLaunchKernel(fn, dim3(qblocks), dim3(128), args, pl->smem_premap4, s) != cudaSuccess)
      return QP_ERR_CUDA;
  } else {
    qpk::premap_fwd_kernel<4><<<pblocks > 0 ? pblocks : 1, 128, 0, s>>>(ma);
  }
  return cuda_status(cudaGetLastError());
}

static void fill_circ(qp_plan* pl, QPCircArgs& a, const WsLayout& w, const float* d_params,
                      const float* const pts[3], const int64_t npts[3], bool grad) {
  char* ws = (char*)pl->ws;
  const int n = pl->c.n_qubits, ppw = geo_ppw(n);
  std::memset(&a, 0, sizeof(a));
  a.s = pl->sched;
  fill_problem(pl, a.pb);
  a.n = n; a.L = pl->c.n_layers; a.m = pl->c.n_readout; a.enc = pl->c.enc;
  a.sstride = grad ? pl->sstride_grad : pl->sstride_fwd;
  int64_t acc = 0, base = 0;
  for (int i = 0; i < 3; ++i) {
    a.pts[i] = pts[i];
    a.npts[i] = npts[i];
    acc += (npts[i] + ppw - 1) / ppw;
    a.task_end[i] = acc;
    a.pt_base[i] = base;
    base += npts[i];
  }
  a.thetaJ = (const float*)(ws + w.thetaJ);
  a.dthetaJ = (float*)(ws + w.dthetaJ);
  a.gates = (const float*)(ws + w.gates);
  a.cenc = (const float*)(ws + w.cenc);
  a.head = d_params + pl->head_off;
  a.counts = (const int32_t*)(ws + w.status) + 1;
  a.blk_loss = (double*)(ws + w.blk_loss);
  a.blk_grad = (float*)(ws + w.blk_grad);
  a.loss_stride = QP_NLP + pl->p.energy_nt;
  a.grad_stride = pl->nE + 3 * pl->c.n_readout + 3;
  a.nE = pl->nE;
  a.nbc = npts[2];
  a.ansatz = pl->c.ansatz;
  a.crz = qp_has_crz(pl->c.ansatz) ? (const float2*)(ws + w.crz) : nullptr;
}

// nblk: block partial slots to sum (-1: the plan's statevector-kernel grid)
static qp_status launch_reduce(qp_plan* pl, const WsLayout& w, const float* d_params, const int64_t npts[3],
                               double* d_loss, float* d_grad, bool mlp, cudaStream_t s, int nsym = 0,
                               int64_t nblk = -1);
// grid_cap > 0: at most that many blocks of the one-pass tensor-core kernel; pdl: launched as the
// programmatic dependent of the kernel before it in the stream
static qp_status launch_premap_bwd(qp_plan* pl, const WsLayout& w, const float* d_params,
                                   const float* const pts[3], const int64_t npts[3], cudaStream_t s,
                                   int grid_cap = 0, bool pdl = false);

// Fused-unitary loss and gradient: forward GEMM per point set, pointwise loss and costates,
// weight-gradient GEMM over all (point, vector) rows, FP64 chunk sum, Y = U' G and the
// B-independent sweep for the Pauli contractions of every gate, then the common reduction.
// With the symmetry penalty (Eq. 18) a fields-only tensor-core pass over the collocation points
// and their mirrors comes first; its per-point cotangents then enter the main pass, the
// mirrored points as rows of set 2 after the boundary points whose cotangents are given.
static qp_status dense_loss_grad(qp_plan* pl, const float* d_params, const float* const pts0[3],
                                 const int64_t npts0[3], double* d_loss, float* d_grad, cudaStream_t s) {
  pl->last_launches = 0;
  const WsLayout w = ws_layout(pl, npts0[0] + npts0[1] + npts0[2]);
  if (!pl->ws || pl->ws_bytes < w.total) return QP_ERR_BUFFER_TOO_SMALL;
  pl->last_stream = s;
  pl->last_status = (const int32_t*)((char*)pl->ws + w.status);
  char* ws = (char*)pl->ws;
  const int n = pl->c.n_qubits, dim = 1 << n, L = pl->c.n_layers;
  int launches = 0;
  const bool sym = pl->p.w_sym > 0.f && npts0[0] > 0;
  const int64_t nm = sym ? (pl->p.medium == QP_MEDIUM_VACUUM ? 2 * npts0[0] : npts0[0]) : 0;
  // the points of the main pass: set 2 extended by the mirrored points
  const float* pts[3] = {pts0[0], pts0[1], sym ? (const float*)(ws + w.sxb) : pts0[2]};
  const int64_t npts[3] = {npts0[0], npts0[1], npts0[2] + nm};
  const int64_t P = npts[0] + npts[1] + npts[2];
  int nsym = 0;
  qpd::BuildArgs ba = {};
  ba.params = d_params; ba.circ_off = pl->circ_off; ba.n = n; ba.L = L;
  ba.gates = (double2*)(ws + w.dgates);
  ba.ansatz = pl->c.ansatz; ba.enc = pl->c.enc; ba.W = (float*)(ws + w.dW); ba.U = (double2*)(ws + w.dU);
  ba.crz64 = qp_has_crz(pl->c.ansatz) ? (const double2*)(ws + w.crz64) : nullptr;
  const bool mlp = pl->c.premap == QP_PREMAP_RFF_MLP;
  const bool fused = fused_path(pl);
  // forward and back-projection on FP16 pairs (the fused n = 7, 8 kernels have no other form)
  const bool fwd16 = fused || pl->operands == QP_OPERANDS_FP16_PAIRS;
  ba.WT = mlp ? (float*)(ws + w.dWT) : nullptr;
  if (mlp && fwd16) {
    ba.WT16 = (__half*)(ws + w.dWT);   // the mu contraction takes FP16 pairs
    ba.WT = nullptr;
  }
  ba.W16 = fwd16 ? (__half*)(ws + w.dW16) : nullptr;
  // the unitary build depends on the circuit parameters only (CRZ ansatze: also on the mesh
  // diagonal of the front launches): it runs on the side stream beside the premap, except
  // with the symmetry penalty, whose fields-only pre-pass needs it first
  const bool side = pl->aux && !qp_has_crz(pl->c.ansatz);
  const bool side_build = side && !sym;
  if (sym) {
    float* xb = (float*)(ws + w.sxb);
    const int64_t tot = npts0[2] + nm;
    qpk::sym_points_kernel<<<(unsigned)((tot + 255) / 256 < pl->sm_count * 4 ? (tot + 255) / 256 : pl->sm_count * 4),
                             256, 0, s>>>(pts0[0], npts0[0], pts0[2], npts0[2], pl->p.medium, xb);
    // fields at the collocation points (set 0) and their mirrors (set 1), no derivatives
    const float* fp[3] = {pts0[0], xb + 3 * npts0[2], nullptr};
    const int64_t fn[3] = {npts0[0], nm, 0};
    qp_status st = launch_front(pl, d_params, fp, fn, w, s, false, true);
    if (st != QP_OK) return st;
    qpd::BuildArgs bp = ba;
    if (fwd16) bp.W = nullptr;
    qpd::dense_gates_kernel<<<1, L * n, 0, s>>>(bp);
    qpd::dense_build_kernel<<<dim, 128, 2 * dim * 16, s>>>(bp);
    qpd::GemmArgs ga = {};
    ga.thetaJ = (const float*)(ws + w.thetaJ); ga.W = (const float*)(ws + w.dW);
    ga.phi = (float2*)(ws + w.dphi); ga.n = n; ga.nv = 1;
    ga.npts = npts0[0] + nm; ga.pt_base = 0; ga.status = (int32_t*)(ws + w.status);
    const int64_t ntiles = (ga.npts + qpd::TM - 1) / qpd::TM;
    const int gblocks = (int)(ntiles < pl->sm_count ? ntiles : pl->sm_count);
    const int64_t items = ntiles * ((2 * dim) / 256);
    const int iblocks = (int)(items < pl->sm_count ? items : pl->sm_count);
    if (fwd16)
      qpd::dense_row16_kernel<0><<<iblocks, qpd::F16_THREADS, qpd::row16_smem_bytes(), s>>>(
          ga, (const __half*)(ws + w.dW16), nullptr);
    else
      qpd::dense_row_gemm_kernel<0><<<gblocks, 128, qpd::gemm_smem_bytes(n, 0), s>>>(ga);
    qpd::ReadoutArgs ra;
    ra.phi = ga.phi; ra.head = d_params + pl->head_off; ra.n = n; ra.m = pl->c.n_readout;
    ra.nv = 1; ra.npts = ga.npts; ra.pt_base = 0; ra.out_f = (float*)(ws + w.sF); ra.out_df = nullptr;
    const int64_t rb = (ga.npts + 7) / 8;
    qpd::dense_readout_kernel<<<(unsigned)(rb < 4096 ? rb : 4096), 256, 0, s>>>(ra);
    const int64_t nb = (npts0[0] + 255) / 256;
    nsym = (int)(nb < pl->sm_count * 4 ? nb : pl->sm_count * 4);
    const double N = (double)(pl->cur_norm[0] > 0 ? pl->cur_norm[0] : npts0[0]);
    qpk::sym_cot_kernel<<<nsym, 256, 0, s>>>((const float*)(ws + w.sF), npts0[0], pl->p.medium, pl->p.w_sym, N,
                                             (float*)(ws + w.sgs), (float*)(ws + w.sge), (double*)(ws + w.spart));
    launches += 7 + front_launches(pl);
  }
  if (side_build) {
    qpd::BuildArgs bs = ba;
    if (fwd16) bs.W = nullptr;
    if (cudaEventRecord(pl->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(pl->aux, pl->ev_fork, 0) != cudaSuccess)
      return QP_ERR_CUDA;
    qpd::dense_gates_kernel<<<1, L * n, 0, pl->aux>>>(bs);
    qpd::dense_build_kernel<<<dim, 128, 2 * dim * 16, pl->aux>>>(bs);
    if (cudaEventRecord(pl->ev_join, pl->aux) != cudaSuccess) return QP_ERR_CUDA;
  }
  qp_status st = launch_front(pl, d_params, pts, npts, w, s, true);
  if (st != QP_OK) return st;
  launches += front_launches(pl);
  if (P > 0 && !front_writes_cs(pl)) {
    const int64_t tot = P * n;
    const int hb = (int)((tot + 255) / 256 < pl->sm_count * 4 ? (tot + 255) / 256 : pl->sm_count * 4);
    qpd::dense_halfangle_kernel<<<hb, 256, 0, s>>>((const float4*)(ws + w.thetaJ), (float2*)(ws + w.dcs), tot);
    launches += 1;
  }
  if (fwd16) ba.W = nullptr;
  if (side_build) {
    if (cudaStreamWaitEvent(s, pl->ev_join, 0) != cudaSuccess) return QP_ERR_CUDA;
    launches += 2;
  } else if (!sym) {
    qpd::dense_gates_kernel<<<1, L * n, 0, s>>>(ba);
    qpd::dense_build_kernel<<<dim, 128, 2 * dim * 16, s>>>(ba);
    launches += 2;
  }
  int64_t base = 0;
  int64_t red_nblk = -1;   // partial slots of the loss and head sums (-1: the plan's block count)
  if (fused) {
    // forward contraction with the pointwise stage as its epilogue (states stay on chip)
    qpd::FusedArgs fa;
    fa.thetaJ = (const float*)(ws + w.thetaJ); fa.W16 = (const __half*)(ws + w.dW16);
    fa.lam = (float*)(ws + w.dphi); fa.rtot = 4 * npts[0] + npts[1] + npts[2];
    fa.head = d_params + pl->head_off;
    fa.n = n; fa.m = pl->c.n_readout;
    for (int i = 0; i < 3; ++i) { fa.pts[i] = pts[i]; fa.npts[i] = npts[i]; fa.pt_base[i] = base; base += npts[i]; }
    fa.tile_end[0] = (npts[0] + 31) / 32;
    fa.tile_end[1] = fa.tile_end[0] + (npts[1] + qpd::TM - 1) / qpd::TM;
    fa.tile_end[2] = fa.tile_end[1] + (npts[2] + qpd::TM - 1) / qpd::TM;
    fill_problem(pl, fa.pb);
    fa.counts = (const int32_t*)(ws + w.status) + 1;
    fa.blk_loss = (double*)(ws + w.blk_loss); fa.blk_grad = (float*)(ws + w.blk_grad);
    fa.loss_stride = QP_NLP + pl->p.energy_nt;
    fa.grad_stride = pl->nE + 3 * pl->c.n_readout + 3;
    fa.nE = pl->nE;
    fa.status = (int32_t*)(ws + w.status);
    fa.scal = (int32_t*)(ws + w.status) + 16;
    fa.wait_limit = pl->wait_limit;
    fa.gsym = sym ? (const float*)(ws + w.sgs) : nullptr;
    fa.gext = sym ? (const float*)(ws + w.sge) : nullptr;
    fa.nbc = npts0[2];
    const int64_t ftiles = fa.tile_end[2];
    const int fblocks = (int)(ftiles < pl->sm_count ? (ftiles > 0 ? ftiles : 1) : pl->sm_count);
    fa.nblk = fblocks;   // one loss/head partial slot per CTA; the reduction sums these only
    red_nblk = fblocks;
    prof_mark(pl, 0, true, s);
    alignas(64) CUtensorMap tmaps[3];
    std::memset(tmaps, 0, sizeof(tmaps));
    fa.use_tma = lam_maps(fa.lam, fa.rtot, npts, (2 * dim) / 256, tmaps) ? 1 : 0;
    const int fsmem = qpd::fused_smem(n, pl->p.energy_nt).total;
    if (n == 7)
      qpd::dense_fused_fwd_kernel<7><<<fblocks, qpd::F_THREADS, fsmem, s>>>(fa, tmaps[0], tmaps[1], tmaps[2]);
    else
      qpd::dense_fused_fwd_kernel<8><<<fblocks, qpd::F_THREADS, fsmem, s>>>(fa, tmaps[0], tmaps[1], tmaps[2]);
    prof_mark(pl, 0, false, s);
    launches += 1;
  } else {
    prof_mark(pl, 0, true, s);
    for (int set = 0; set < 3; ++set) {
      if (npts[set] > 0) {
        qpd::GemmArgs ga = {};
        ga.thetaJ = (const float*)(ws + w.thetaJ); ga.W = (const float*)(ws + w.dW);
        ga.phi = (float2*)(ws + w.dphi); ga.n = n; ga.nv = set == 0 ? 4 : 1;
        ga.npts = npts[set]; ga.pt_base = base; ga.status = (int32_t*)(ws + w.status);
        ga.cs = (const float2*)(ws + w.dcs);   // half-angle factors of the call
        const int64_t ppt = qpd::TM / ga.nv;
        const int64_t ntiles = (npts[set] + ppt - 1) / ppt;
        const int gblocks = (int)(ntiles < pl->sm_count ? ntiles : pl->sm_count);
        const int64_t items = ntiles * ((2 * dim) / 256);   // (tile, column chunk) items
        const int iblocks = (int)(items < pl->sm_count ? items : pl->sm_count);
        if (fwd16)   // records the operand range of R for the weight gradient
          qpd::dense_row16_kernel<0><<<iblocks, qpd::F16_THREADS, qpd::row16_smem_bytes(), s>>>(
              ga, (const __half*)(ws + w.dW16), (int32_t*)(ws + w.status) + 16);
        else
          qpd::dense_row_gemm_kernel<0><<<gblocks, 128, qpd::gemm_smem_bytes(n, 0), s>>>(ga);
        launches += 1;
      }
      base += npts[set];
    }
    prof_mark(pl, 0, false, s);
    qpd::PointArgs pa;
    pa.phi = (float2*)(ws + w.dphi); pa.head = d_params + pl->head_off; pa.n = n; pa.m = pl->c.n_readout;
    base = 0;
    for (int i = 0; i < 3; ++i) { pa.pts[i] = pts[i]; pa.npts[i] = npts[i]; pa.pt_base[i] = base; base += npts[i]; }
    fill_problem(pl, pa.pb);
    pa.counts = (const int32_t*)(ws + w.status) + 1;
    pa.blk_loss = (double*)(ws + w.blk_loss); pa.blk_grad = (float*)(ws + w.blk_grad);
    pa.loss_stride = QP_NLP + pl->p.energy_nt;
    pa.grad_stride = pl->nE + 3 * pl->c.n_readout + 3;
    pa.nE = pl->nE;
    pa.lmax = fwd16 ? (int32_t*)(ws + w.status) + 17 : nullptr;   // scale of the mu operand
    pa.gsym = sym ? (const float*)(ws + w.sgs) : nullptr;
    pa.gext = sym ? (const float*)(ws + w.sge) : nullptr;
    pa.nbc = npts0[2];
    const int psmem = ((QP_NLP + pl->p.energy_nt) * 8 + 15) / 16 * 16 + (3 * pl->c.n_readout + 3) * 4;
    if (n == 9)
      qpd::dense_point_kernel<9><<<pl->blocks_grad, qpd::PT_POINT_THREADS, psmem, s>>>(pa);
    else
      qpd::dense_point_kernel<10><<<pl->blocks_grad, qpd::PT_POINT_THREADS, psmem, s>>>(pa);
    launches += 1;
  }
  qpd::WgArgs wa;
  wa.thetaJ = (const float*)(ws + w.thetaJ); wa.cs = (const float2*)(ws + w.dcs);
  wa.lam = (const float*)(ws + w.dphi);
  wa.rtot = fused ? 4 * npts[0] + npts[1] + npts[2] : 0;
  wa.part = (float*)(ws + w.dpart); wa.n = n;
  base = 0;
  for (int i = 0; i < 3; ++i) { wa.npts[i] = npts[i]; wa.pt_base[i] = base; base += npts[i]; }
  wa.kc_end[0] = (4 * npts[0] + qpd::WKC - 1) / qpd::WKC;
  wa.kc_end[1] = wa.kc_end[0] + (npts[1] + qpd::WKC - 1) / qpd::WKC;
  wa.kc_end[2] = wa.kc_end[1] + (npts[2] + qpd::WKC - 1) / qpd::WKC;
  const WgGeom wgm = wg_geom(pl, wa.kc_end[2]);
  if (wgm.nslots > wg_slots_cap(pl)) return QP_ERR_INTERNAL;
  if ((int64_t)wgm.tiles * wa.kc_end[2] > (int64_t)INT32_MAX) return QP_ERR_UNSUPPORTED;   // 32-bit step counts
  wa.tiles = wgm.tiles; wa.nslots = (int32_t)wgm.nslots; wa.fl = wgm.fl;
  wa.status = (int32_t*)(ws + w.status);
  prof_mark(pl, 1, true, s);
  wa.scal = (const int32_t*)(ws + w.status) + 16;
  {
    // FP16 pairs when the forward recorded both operand ranges
    void* wargs[] = {&wa};
    const cudaError_t le = cudaLaunchKernel(fwd16 ? wgrad_kernel<true>(n) : wgrad_kernel<false>(n),
                                            dim3((unsigned)wgm.grid), dim3(qpd::wgc_threads(fwd16)),
                                            wargs, qpd::wgc_smem(n, fwd16).total, s);
    if (le != cudaSuccess) return QP_ERR_CUDA;
  }
  prof_mark(pl, 1, false, s);
  launches += 1;
  // the gate-gradient chain (slot sum, Y = U'G, sweep) depends on G only: on the side stream,
  // beside mu and the premap backward, joined back before the reduction. With the one-pass
  // premap backward (n = 7, 8) the chain stops at Y on the side stream; the sweep cluster runs
  // on the call's stream after mu, and the premap backward is launched as its programmatic
  // dependent on the other SMs (a one-wave kernel started first would hold every SM, and the
  // cluster would wait for it to drain).
  const bool pdl_tail = side && fused && mlp && !pl->deep && pl->pg_ok;
  const int sweep_S = qpd::swc_size(n, pl->swc_big);
  cudaStream_t ss = s;
  if (side) {
    if (cudaEventRecord(pl->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(pl->aux, pl->ev_fork, 0) != cudaSuccess)
      return QP_ERR_CUDA;
    ss = pl->aux;
  }
  qpd::SweepArgs sa;
  sa.part = wa.part; sa.nchunks = (int32_t)wgm.nslots; sa.n = n; sa.L = L; sa.ansatz = pl->c.ansatz;
  sa.U = (const double2*)(ws + w.dU); sa.G = (float2*)(ws + w.dG); sa.Y = (float2*)(ws + w.dY);
  sa.params = d_params; sa.circ_off = pl->circ_off; sa.eout = (float*)(ws + w.blk_grad);
  sa.gates = (const double2*)(ws + w.dgates);
  sa.crz = qp_has_crz(pl->c.ansatz) ? (const float2*)(ws + w.crz) : nullptr;
  {
    const int gg = gsum_groups(pl);
    qpd::dense_gsum_kernel<<<dim3((dim * dim + 255) / 256, gg), 256, 0, ss>>>(sa, gg, (float4*)(ws + w.dgs));
    const int64_t fb = ((int64_t)dim * dim + 255) / 256;
    qpd::dense_gsum_fin_kernel<<<(unsigned)(fb < pl->sm_count * 8 ? fb : pl->sm_count * 8), 256, 0, ss>>>(
        sa, gg, (const float4*)(ws + w.dgs));
    launches += 1;
  }
  qpd::dense_y_kernel<<<dim3(dim / 16, dim / 16), 256, 0, ss>>>(sa);
  // the whole sweep in one cluster launch (Y lives in the cluster's shared memory), n <= 8
  auto launch_sweep = [&](cudaStream_t st) -> qp_status {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sweep_S);
    cfg.blockDim = dim3(qpd::SWC_THREADS);
    cfg.dynamicSmemBytes = qpd::swc_smem(n, L, sweep_S, qp_crz_sums(pl->c.ansatz, n));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = sweep_S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, qpd::dense_sweep_cluster_kernel, sa) != cudaSuccess ? QP_ERR_CUDA : QP_OK;
  };
  if (n <= 8) {
    if (!pdl_tail) {
      const qp_status sst = launch_sweep(ss);
      if (sst != QP_OK) return sst;
    }
    launches += 1;
  } else {
    float2* Ya = sa.Y;
    float2* Yb = sa.G;  // the G scratch is free once Y = U' G is formed
    const int tcol = 16, trow = 16;
    const int64_t tot = (int64_t)dim * dim;
    const int rblocks = (int)((tot + 255) / 256 < pl->sm_count * 8 ? (tot + 255) / 256 : pl->sm_count * 8);
    for (int l = L - 1; l >= 0; --l) {
      qpd::dense_sweep_ring_kernel<<<rblocks, 256, 0, ss>>>(sa, l, Ya, Yb);
      if (l > 0) {
        qpd::dense_sweep_left_kernel<16><<<dim / tcol, 256, dim * tcol * 8, ss>>>(sa, l, Yb);
        qpd::dense_sweep_right_kernel<16><<<dim / trow, 256, dim * trow * 8, ss>>>(sa, l, Yb);
        launches += 2;
      }
      float2* t = Ya; Ya = Yb; Yb = t;
      launches += 1;
    }
  }
  launches += 2;
  if (side && cudaEventRecord(pl->ev_join, pl->aux) != cudaSuccess) return QP_ERR_CUDA;
  if (mlp) {
    if (fused) {
      // mu rows on the tensor cores with the embedding gradients as the epilogue
      qpd::MuArgs ma;
      ma.thetaJ = (const float*)(ws + w.thetaJ); ma.WT16 = (const __half*)(ws + w.dWT);
      ma.scal = (const int32_t*)(ws + w.status) + 16;
      ma.lam = (const float*)(ws + w.dphi); ma.rtot = 4 * npts[0] + npts[1] + npts[2];
      ma.dthetaJ = (float*)(ws + w.dthetaJ); ma.n = n;
      base = 0;
      for (int i = 0; i < 3; ++i) { ma.npts[i] = npts[i]; ma.pt_base[i] = base; base += npts[i]; }
      ma.tile_end[0] = (npts[0] + 31) / 32;
      ma.tile_end[1] = ma.tile_end[0] + (npts[1] + qpd::TM - 1) / qpd::TM;
      ma.tile_end[2] = ma.tile_end[1] + (npts[2] + qpd::TM - 1) / qpd::TM;
      ma.status = (int32_t*)(ws + w.status);
      const int64_t mt = ma.tile_end[2];
      const int mblocks = (int)(mt < pl->sm_count ? (mt > 0 ? mt : 1) : pl->sm_count);
      prof_mark(pl, 2, true, s);
      if (n == 7)
        qpd::dense_mu_embed_kernel<7><<<mblocks, qpd::MU_THREADS, qpd::mu_smem_bytes(n), s>>>(ma);
      else
        qpd::dense_mu_embed_kernel<8><<<mblocks, qpd::MU_THREADS, qpd::mu_smem_bytes(n), s>>>(ma);
      prof_mark(pl, 2, false, s);
      launches += 1;
    } else {
      // back-projection mu = Re(U'^H lambda) per (point, vector) row, then the embedding
      // gradients per point, then the premap backward shared with the SIMT path
      base = 0;
      prof_mark(pl, 2, true, s);
      for (int set = 0; set < 3; ++set) {
        if (npts[set] > 0) {
          qpd::GemmArgs ga = {};
          ga.thetaJ = (const float*)(ws + w.thetaJ); ga.W = (const float*)(ws + w.dWT);
          ga.phi = nullptr; ga.lam = (const float*)(ws + w.dphi); ga.mu = (float*)(ws + w.dmu);
          ga.n = n; ga.nv = set == 0 ? 4 : 1;
          ga.npts = npts[set]; ga.pt_base = base; ga.status = (int32_t*)(ws + w.status);
          const int64_t ppt = qpd::TM / ga.nv;
          const int64_t ntiles = (npts[set] + ppt - 1) / ppt;
          const int gblocks = (int)(ntiles < pl->sm_count ? ntiles : pl->sm_count);
          const int64_t items = ntiles * (dim / 256);   // (tile, column chunk) items
          const int iblocks = (int)(items < pl->sm_count ? items : pl->sm_count);
          if (fwd16)
            qpd::dense_row16_kernel<1><<<iblocks, qpd::F16_THREADS, qpd::row16_smem_bytes(), s>>>(
                ga, (const __half*)(ws + w.dWT), (int32_t*)(ws + w.status) + 16);
          else
            qpd::dense_row_gemm_kernel<1><<<gblocks, 128, qpd::gemm_smem_bytes(n, 1), s>>>(ga);
          launches += 1;
        }
        base += npts[set];
      }
      prof_mark(pl, 2, false, s);
      qpd::EmbedArgs ea;
      ea.thetaJ = (const float*)(ws + w.thetaJ); ea.mu = (const float*)(ws + w.dmu);
      ea.dthetaJ = (float*)(ws + w.dthetaJ); ea.n = n; ea.cs = (const float2*)(ws + w.dcs);
      base = 0;
      for (int i = 0; i < 3; ++i) { ea.npts[i] = npts[i]; ea.pt_base[i] = base; base += npts[i]; }
      const int64_t eb = (P + 7) / 8;
      qpd::dense_embed_grad_kernel<<<(unsigned)(eb < 8192 ? eb : 8192), 256, 0, s>>>(ea);
      launches += 1;
    }
    if (pdl_tail) {
      // Y is ready on the side stream: the sweep on this stream, then the premap backward on
      // the SMs the sweep cluster leaves (two blocks per SM)
      if (cudaStreamWaitEvent(s, pl->ev_join, 0) != cudaSuccess) return QP_ERR_CUDA;
      st = launch_sweep(s);
      if (st != QP_OK) return st;
      st = launch_premap_bwd(pl, w, d_params, pts, npts, s, 2 * (pl->sm_count - sweep_S), true);
    } else {
      st = launch_premap_bwd(pl, w, d_params, pts, npts, s);
    }
    if (st != QP_OK) return st;
    launches += premap_bwd_launches(pl);
  }
  if (side && !pdl_tail && cudaStreamWaitEvent(s, pl->ev_join, 0) != cudaSuccess) return QP_ERR_CUDA;
  st = launch_reduce(pl, w, d_params, npts0, d_loss, d_grad, mlp, s, nsym, red_nblk);
  pl->last_launches = launches + 1;
  return st;
}

qp_status qp_forward(qp_plan* pl, const float* d_params, const float* d_pts, int64_t B,
                     float* d_fields, float* d_dfields, void* stream) {
  if (!pl || !d_params || B < 0 || (B > 0 && (!d_pts || !d_fields))) return QP_ERR_INVALID_ARG;
  pl->cur_norm[0] = pl->cur_norm[1] = pl->cur_norm[2] = 0;
  pl->cur_norm_diel = pl->cur_colloc_off = 0;
  pl->last_launches = 0;
  if (B == 0) return QP_OK;
  const WsLayout w = ws_layout(pl, B);
  if (!pl->ws || pl->ws_bytes < w.total) return QP_ERR_BUFFER_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  pl->last_stream = s;
  pl->last_status = (const int32_t*)((char*)pl->ws + w.status);
  const float* pts[3] = {d_pts, nullptr, nullptr};
  const int64_t npts[3] = {B, 0, 0};
  qp_status st = launch_front(pl, d_params, pts, npts, w, s, false, d_dfields == nullptr);
  if (st != QP_OK) return st;
  if (dense_path(pl)) {
    char* ws = (char*)pl->ws;
    const int n = pl->c.n_qubits, dim = 1 << n;
    qpd::BuildArgs ba = {};
    ba.params = d_params; ba.circ_off = pl->circ_off; ba.n = n; ba.L = pl->c.n_layers;
    ba.ansatz = pl->c.ansatz; ba.enc = pl->c.enc; ba.W = (float*)(ws + w.dW); ba.U = nullptr;
    ba.crz64 = qp_has_crz(pl->c.ansatz) ? (const double2*)(ws + w.crz64) : nullptr;
    const bool fwd16 = n >= 7 && pl->operands == QP_OPERANDS_FP16_PAIRS;
    ba.W16 = fwd16 ? (__half*)(ws + w.dW16) : nullptr;
    if (fwd16) ba.W = nullptr;
    ba.gates = (double2*)(ws + w.dgates);
    qpd::dense_gates_kernel<<<1, pl->c.n_layers * n, 0, s>>>(ba);
    qpd::dense_build_kernel<<<dim, 128, 2 * dim * 16, s>>>(ba);
    qpd::GemmArgs ga = {};
    ga.thetaJ = (const float*)(ws + w.thetaJ); ga.W = (const float*)(ws + w.dW);
    ga.phi = (float2*)(ws + w.dphi); ga.n = n; ga.nv = d_dfields ? 4 : 1;
    ga.npts = B; ga.pt_base = 0; ga.status = (int32_t*)(ws + w.status);
    const int64_t ppt = qpd::TM / ga.nv;
    const int64_t ntiles = (B + ppt - 1) / ppt;
    const int gblocks = (int)(ntiles < pl->sm_count ? ntiles : pl->sm_count);
    const int64_t items = ntiles * ((2 * dim) / 256);   // (tile, column chunk) items
    const int iblocks = (int)(items < pl->sm_count ? items : pl->sm_count);
    prof_mark(pl, 0, true, s);
    if (fwd16)
      qpd::dense_row16_kernel<0><<<iblocks, qpd::F16_THREADS, qpd::row16_smem_bytes(), s>>>(
          ga, (const __half*)(ws + w.dW16), nullptr);
    else
      qpd::dense_row_gemm_kernel<0><<<gblocks, 128, qpd::gemm_smem_bytes(n, 0), s>>>(ga);
    prof_mark(pl, 0, false, s);
    qpd::ReadoutArgs ra;
    ra.phi = ga.phi; ra.head = d_params + pl->head_off; ra.n = n; ra.m = pl->c.n_readout;
    ra.nv = ga.nv; ra.npts = B; ra.pt_base = 0; ra.out_f = d_fields; ra.out_df = d_dfields;
    const int64_t rb = (B + 7) / 8;
    qpd::dense_readout_kernel<<<(unsigned)(rb < 4096 ? rb : 4096), 256, 0, s>>>(ra);
    pl->last_launches = front_launches(pl) + 3;
    return cuda_status(cudaGetLastError());
  }
  QPCircArgs a;
  fill_circ(pl, a, w, d_params, pts, npts, false);
  a.want_df = d_dfields != nullptr;
  a.out_f = d_fields;
  a.out_df = d_dfields;
  const int64_t tasks = a.task_end[2];
  int64_t blocks = (tasks + pl->warps_fwd - 1) / pl->warps_fwd;
  if (blocks > pl->blocks_fwd) blocks = pl->blocks_fwd;
  void* args[] = {&a};
  prof_mark(pl, 0, true, s);
  if (cudaLaunchKernel(circuit_kernel_ptr(pl->c.n_qubits, false, qp_has_crz(pl->c.ansatz)), dim3((unsigned)blocks),
                       dim3(pl->warps_fwd * 32), args, pl->smem_fwd, s) != cudaSuccess)
    return QP_ERR_CUDA;
  prof_mark(pl, 0, false, s);
  pl->last_launches = front_launches(pl) + 1;
  return cuda_status(cudaGetLastError());
}

// Argument checks of a loss call (nothing launched, no plan state changed).
static qp_status check_loss_args(const qp_plan* pl, const float* d_params, const qp_batch* batch,
                                 const double* d_loss, const float* d_grad) {
  if (!pl || !d_params || !batch || !d_loss || !d_grad) return QP_ERR_INVALID_ARG;
  if (batch->n_colloc < 0 || batch->n_ic < 0 || batch->n_bc < 0) return QP_ERR_INVALID_ARG;
  if ((batch->n_colloc && !batch->colloc) || (batch->n_ic && !batch->ic) || (batch->n_bc && !batch->bc))
    return QP_ERR_INVALID_ARG;
  // sharding fields: whole-loss counts cover this call's sets, the offset places its
  // collocation points inside the whole set
  const int64_t nloc[3] = {batch->n_colloc, batch->n_ic, batch->n_bc};
  const int64_t nrm[3] = {batch->norm_colloc, batch->norm_ic, batch->norm_bc};
  for (int i = 0; i < 3; ++i)
    if (nrm[i] < 0 || (nrm[i] > 0 && nrm[i] < nloc[i])) return QP_ERR_INVALID_ARG;
  if (batch->colloc_offset < 0) return QP_ERR_INVALID_ARG;
  if (nrm[0] > 0 && (batch->norm_diel < 0 || batch->norm_diel > nrm[0] ||
                     batch->colloc_offset + batch->n_colloc > nrm[0]))
    return QP_ERR_INVALID_ARG;
  if (nrm[0] == 0 && batch->colloc_offset != 0) return QP_ERR_INVALID_ARG;
  if (dense_path(pl) && pl->c.n_qubits < 7) return QP_ERR_UNSUPPORTED;
  const int64_t P = nloc[0] + nloc[1] + nloc[2];
  if (!pl->ws || pl->ws_bytes < ws_layout(pl, P).total) return QP_ERR_BUFFER_TOO_SMALL;
  return QP_OK;
}

qp_status qp_loss_grad(qp_plan* pl, const float* d_params, const qp_batch* batch, double* d_loss,
                       float* d_grad, void* stream) {
  const qp_status chk = check_loss_args(pl, d_params, batch, d_loss, d_grad);
  if (chk != QP_OK) return chk;
  const int64_t nrm[3] = {batch->norm_colloc, batch->norm_ic, batch->norm_bc};
  for (int i = 0; i < 3; ++i) pl->cur_norm[i] = nrm[i];
  pl->cur_norm_diel = nrm[0] > 0 ? batch->norm_diel : 0;
  pl->cur_colloc_off = batch->colloc_offset;
  pl->last_launches = 0;
  const float* pts[3] = {batch->colloc, batch->ic, batch->bc};
  if (dense_path(pl)) {
    if (pl->c.n_qubits < 7) return QP_ERR_UNSUPPORTED;
    const int64_t np3[3] = {batch->n_colloc, batch->n_ic, batch->n_bc};
    return dense_loss_grad(pl, d_params, pts, np3, d_loss, d_grad, (cudaStream_t)stream);
  }
  const int64_t npts[3] = {batch->n_colloc, batch->n_ic, batch->n_bc};
  const int64_t P = npts[0] + npts[1] + npts[2];
  const WsLayout w = ws_layout(pl, P);
  if (!pl->ws || pl->ws_bytes < w.total) return QP_ERR_BUFFER_TOO_SMALL;
  cudaStream_t s = (cudaStream_t)stream;
  pl->last_stream = s;
  pl->last_status = (const int32_t*)((char*)pl->ws + w.status);
  char* ws = (char*)pl->ws;
  int launches = 0;
  // symmetry penalty (Eq. 18): fields at the collocation points and their mirrors first, then
  // the main pass with the mirrored points appended to set 2 as given-cotangent rows
  const bool sym = pl->p.w_sym > 0.f && npts[0] > 0;
  const int64_t nm = sym ? (pl->p.medium == QP_MEDIUM_VACUUM ? 2 * npts[0] : npts[0]) : 0;
  int nsym = 0;
  const float* mpts[3] = {pts[0], pts[1], pts[2]};
  int64_t mnp[3] = {npts[0], npts[1], npts[2]};
  if (sym) {
    float* xb = (float*)(ws + w.sxb);
    const int64_t tot = npts[2] + nm;
    qpk::sym_points_kernel<<<(unsigned)((tot + 255) / 256 < pl->sm_count * 4 ? (tot + 255) / 256 : pl->sm_count * 4),
                             256, 0, s>>>(pts[0], npts[0], pts[2], npts[2], pl->p.medium, xb);
    const float* fp[3] = {pts[0], xb + 3 * npts[2], nullptr};
    const int64_t fn[3] = {npts[0], nm, 0};
    qp_status st = launch_front(pl, d_params, fp, fn, w, s, false, true);
    if (st != QP_OK) return st;
    QPCircArgs fa;
    fill_circ(pl, fa, w, d_params, fp, fn, false);
    fa.want_df = 0;
    fa.out_f = (float*)(ws + w.sF);
    const int64_t ftasks = fa.task_end[2];
    int64_t fblocks = (ftasks + pl->warps_fwd - 1) / pl->warps_fwd;
    if (fblocks > pl->blocks_fwd) fblocks = pl->blocks_fwd;
    void* fargs[] = {&fa};
    if (cudaLaunchKernel(circuit_kernel_ptr(pl->c.n_qubits, false, qp_has_crz(pl->c.ansatz)), dim3((unsigned)fblocks),
                         dim3(pl->warps_fwd * 32), fargs, pl->smem_fwd, s) != cudaSuccess)
      return QP_ERR_CUDA;
    const int64_t nb = (npts[0] + 255) / 256;
    nsym = (int)(nb < pl->sm_count * 4 ? nb : pl->sm_count * 4);
    const double N = (double)(pl->cur_norm[0] > 0 ? pl->cur_norm[0] : npts[0]);
    qpk::sym_cot_kernel<<<nsym, 256, 0, s>>>((const float*)(ws + w.sF), npts[0], pl->p.medium, pl->p.w_sym, N,
                                             (float*)(ws + w.sgs), (float*)(ws + w.sge), (double*)(ws + w.spart));
    launches += 3 + front_launches(pl);
    mpts[2] = xb;
    mnp[2] = npts[2] + nm;
  }
  if (P > 0) {
    qp_status st = launch_front(pl, d_params, mpts, mnp, w, s, true);
    if (st != QP_OK) return st;
    launches += front_launches(pl);
  } else {
    // nothing to evaluate: still clear the status/counters through the prep kernel
    qpk::PrepArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.params = d_params; pa.circ_off = pl->circ_off; pa.n = pl->c.n_qubits; pa.L = pl->c.n_layers;
    pa.ansatz = pl->c.ansatz; pa.enc = pl->c.enc;
    pa.gates = (float*)(ws + w.gates); pa.cmat = (float*)(ws + w.cmat); pa.cenc = (float*)(ws + w.cenc);
    pa.counts = (int32_t*)(ws + w.status) + 1; pa.status = (int32_t*)(ws + w.status);
    qpk::prep_kernel<<<(pa.L * pa.n + 63) / 64, 64, 0, s>>>(pa);
    launches += 1;
  }
  QPCircArgs a;
  fill_circ(pl, a, w, d_params, mpts, mnp, true);
  if (sym) {
    a.gsym = (const float*)(ws + w.sgs);
    a.gext = (const float*)(ws + w.sge);
    a.nbc = npts[2];
  }
  const bool mlp = pl->c.premap == QP_PREMAP_RFF_MLP;
  a.want_dtheta = mlp ? 1 : 0;
  const int64_t tasks = a.task_end[2];
  // every block writes its partials, so the grid is fixed to the plan's block count
  void* args[] = {&a};
  prof_mark(pl, 0, true, s);
  if (cudaLaunchKernel(circuit_kernel_ptr(pl->c.n_qubits, true, qp_has_crz(pl->c.ansatz)), dim3(pl->blocks_grad),
                       dim3(pl->warps_grad * 32), args, pl->smem_grad, s) != cudaSuccess)
    return QP_ERR_CUDA;
  prof_mark(pl, 0, false, s);
  (void)tasks;
  launches += 1;
  if (mlp) {
    qp_status stb = launch_premap_bwd(pl, w, d_params, mpts, mnp, s);
    if (stb != QP_OK) return stb;
    launches += premap_bwd_launches(pl);
  }
  qp_status st_red;
  st_red = launch_reduce(pl, w, d_params, npts, d_loss, d_grad, mlp, s, nsym);
  pl->last_launches = launches + 1;
  return st_red;
}

// Premap backward (per point) and its weight-gradient partials, from dL/dtheta and dL/dJ.
static qp_status launch_premap_bwd(qp_plan* pl, const WsLayout& w, const float* d_params,
                                   const float* const pts[3], const int64_t npts[3], cudaStream_t s,
                                   int grid_cap, bool pdl) {
  char* ws = (char*)pl->ws;
  pl->wblk = pl->nwblk;
  const int64_t P = npts[0] + npts[1] + npts[2];
  qpk::PremapArgs ma;
  std::memset(&ma, 0, sizeof(ma));
  for (int i = 0; i < 3; ++i) { ma.pts[i] = pts[i]; ma.npts[i] = npts[i]; }
  ma.ptot = P;
  ma.params = d_params; ma.n = pl->c.n_qubits; ma.premap = pl->c.premap; ma.scale = pl->c.scale;
  ma.F = pl->c.rff_freqs; ma.H = pl->c.mlp_width;
  ma.thetaJ = (float*)(ws + w.thetaJ);
  ma.dthetaJ = (const float*)(ws + w.dthetaJ);
  ma.d1 = (float*)(ws + w.d1); ma.d2 = (float*)(ws + w.d2); ma.u1 = (float*)(ws + w.u1);
  if (pl->deep) return launch_mlp_bwd(pl, d_params, pts, npts, w, s);
  if (pl->pg_ok) {
    // backward and weight-gradient partials in one pass (one partial slot per block)
    ma.status = (int32_t*)(ws + w.status);
    const int grid = grid_cap > 0 && grid_cap < pl->nwblk ? grid_cap : pl->nwblk;
    pl->wblk = grid;   // the reduction sums exactly the slots written
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(qpk::PG_THREADS);
    cfg.dynamicSmemBytes = qpk::pb_smem(pl->c.n_qubits);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cuda_status(cudaLaunchKernelEx(&cfg, qpk::premap_bwd_tc_kernel, ma, (float*)(ws + w.wpart),
                                          (int32_t)(pl->mlp_count - pl->nfixed)));
  }
  if (P > 0) {
    const int64_t qb = (P + 31) / 32;
    const int pblocks = (int)(qb < pl->sm_count * 8 ? qb : pl->sm_count * 8);
    void* bargs[] = {&ma};
    if (cudaLaunchKernel(premap_bwd4_ptr(pl->c.mlp_width), dim3(pblocks), dim3(128), bargs,
                         pl->smem_premap4, s) != cudaSuccess)
      return QP_ERR_CUDA;
  }
  qpk::WgradArgs wa;
  wa.p = ma;
  wa.part = (float*)(ws + w.wpart);
  wa.nW = (int32_t)(pl->mlp_count - pl->nfixed);
  wa.tile = pl->wtile;
  void* wargs[] = {&wa};
  if (cudaLaunchKernel((void*)qpk::premap_wgrad_kernel, dim3(pl->nwblk), dim3(256), wargs,
                       pl->smem_wgrad, s) != cudaSuccess)
    return QP_ERR_CUDA;
  return cuda_status(cudaGetLastError());
}

static qp_status launch_reduce(qp_plan* pl, const WsLayout& w, const float* d_params, const int64_t npts[3],
                               double* d_loss, float* d_grad, bool mlp, cudaStream_t s, int nsym,
                               int64_t nblk) {
  char* ws = (char*)pl->ws;
  qpk::ReduceArgs ra;
  ra.sym_part = nsym > 0 ? (const double*)(ws + w.spart) : nullptr;
  ra.nsym = nsym;
  ra.w_sym = pl->p.w_sym;
  ra.blk_loss = (const double*)(ws + w.blk_loss);
  ra.blk_grad = (const float*)(ws + w.blk_grad);
  ra.nblk = nblk >= 0 ? (int32_t)nblk : pl->blocks_grad;
  ra.loss_stride = QP_NLP + pl->p.energy_nt;
  ra.grad_stride = pl->nE + 3 * pl->c.n_readout + 3;
  ra.nE = pl->nE;
  ra.ansatz = pl->c.ansatz;
  ra.wpart = (const float*)(ws + w.wpart);
  ra.nwblk = mlp ? pl->wblk : 0;
  ra.nW = (int32_t)(pl->mlp_count - pl->nfixed);
  ra.cmat = (const float*)(ws + w.cmat);
  ra.counts = (const int32_t*)(ws + w.status) + 1;
  ra.status = (int32_t*)(ws + w.status);
  ra.loss = d_loss; ra.grad = d_grad;
  ra.nparams = pl->n_params; ra.circ_off = pl->circ_off; ra.head_off = pl->head_off;
  ra.mlp_off = pl->nfixed; ra.mlp_count = pl->mlp_count - pl->nfixed;
  ra.n = pl->c.n_qubits; ra.L = pl->c.n_layers; ra.m = pl->c.n_readout;
  ra.k = qp_ansatz_k(pl->c.ansatz);
  ra.nt = pl->p.energy_nt; ra.medium = pl->p.medium; ra.phys_loss = pl->p.phys_loss;
  ra.nc = pl->cur_norm[0] > 0 ? pl->cur_norm[0] : npts[0];
  ra.ni = pl->cur_norm[1] > 0 ? pl->cur_norm[1] : npts[1];
  ra.nb = pl->cur_norm[2] > 0 ? pl->cur_norm[2] : npts[2];
  ra.norm_diel = pl->cur_norm[0] > 0 ? pl->cur_norm_diel : -1;
  ra.w_ic = pl->p.w_ic; ra.w_bc = pl->p.w_bc; ra.w_energy = pl->p.w_energy;
  const int64_t nwarps = pl->n_params + 1 + ra.nt;   // one warp per output
  ra.nmain_blocks = (int32_t)((nwarps + 7) / 8);
  ra.mlp_blocks = ra.mlp_count > 0 ? (int32_t)((ra.mlp_count + 31) / 32) : 0;
  qpk::reduce_kernel<<<(unsigned)(ra.nmain_blocks + ra.mlp_blocks), 256, 0, s>>>(ra);
  return cuda_status(cudaGetLastError());
}

qp_status qp_last_device_error(qp_plan* pl) {
  if (!pl) return QP_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(pl->last_stream) != cudaSuccess) return QP_ERR_CUDA;
  if (!pl->last_status) return QP_OK;
  int32_t st = 0;
  if (cudaMemcpy(&st, pl->last_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return QP_ERR_CUDA;
  return (qp_status)st;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Allocation-free forward call (qp_forward_noalloc).
//
// Some callers cannot allocate device memory at all: code running inside a memory pool that
// refuses new allocations, plugins handed a fixed device budget, or hosts where cudaMalloc is
// not allowed after start-up. For them the scratch of the forward call (gate tables and the
// per-point angles and input Jacobian) lives in one fixed array of device memory that belongs
// to the library. Every GPU that loads the library holds this array until the process exits.
#include <mutex>

static constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char qp_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the fixed scratch on the current device. In host code the array's name is
// only a stand-in, so the real address comes from cudaGetSymbolAddress with the device current.
// It is looked up again on every call made outside stream capture, so it follows the module
// when the device's context is re-created; a call made while `s` is capturing uses the address
// of the last call outside capture on this device (and fails if there was none).
qp_status noalloc_scratch_address(cudaStream_t s, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return QP_ERR_CUDA; }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return QP_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) { cudaGetLastError(); return QP_ERR_CUDA; }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, qp_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return QP_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  } else if (!g_noalloc_addr[dev]) {
    return QP_ERR_CUDA;
  }
  *out = g_noalloc_addr[dev];
  return QP_OK;
}
}  // namespace

qp_status qp_count_dielectric(qp_plan* pl, const float* d_pts, int64_t n, int64_t* d_count, void* stream) {
  if (!pl || !d_count || n < 0 || (n > 0 && !d_pts)) return QP_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_count, 0, sizeof(int64_t), s) != cudaSuccess) return QP_ERR_CUDA;
  pl->last_launches = 0;
  if (n > 0 && pl->p.medium == QP_MEDIUM_DIELECTRIC) {
    const int64_t nb = (n + 255) / 256;
    qpk::count_dielectric_kernel<<<(unsigned)(nb < pl->sm_count * 4 ? nb : pl->sm_count * 4), 256, 0, s>>>(
        d_pts, n, pl->p.disk_x0, pl->p.disk_y0, pl->p.disk_r, reinterpret_cast<unsigned long long*>(d_count));
    if (cudaGetLastError() != cudaSuccess) return QP_ERR_CUDA;
    pl->last_launches = 1;
  }
  return QP_OK;
}

namespace {
// Library-owned worker streams of qp_batch_step, created once per device.
constexpr int QP_BATCH_STREAMS = 8;
constexpr int QP_GROUP_STREAMS = 4;   // streams of the multi-instance launches (one per qubit count in turn)
struct BatchStreams {
  cudaStream_t st[QP_BATCH_STREAMS];
  cudaEvent_t fork, join[QP_BATCH_STREAMS];
  cudaStream_t gst[QP_GROUP_STREAMS];
  cudaEvent_t gfork, gjoin[QP_GROUP_STREAMS];
  bool ok = false;
};
std::mutex g_batch_mu;
BatchStreams g_batch[64];

BatchStreams* batch_streams() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchStreams& b = g_batch[dev];
  if (!b.ok) {
    for (int i = 0; i < QP_BATCH_STREAMS; ++i) {
      if (cudaStreamCreateWithFlags(&b.st[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
      if (cudaEventCreateWithFlags(&b.join[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    if (cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    for (int i = 0; i < QP_GROUP_STREAMS; ++i) {
      if (cudaStreamCreateWithFlags(&b.gst[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
      if (cudaEventCreateWithFlags(&b.gjoin[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    if (cudaEventCreateWithFlags(&b.gfork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    b.ok = true;
  }
  return &b;
}
}  // namespace

// ---------------------------------------------------------------- multi-instance launch
namespace {
constexpr int kMultiK[3] = {1, 4, 16};      // tuner candidates: tasks per item = warps x K
constexpr int kMultiW[3] = {4, 8, 12};      // tuner candidates: warps per CTA
constexpr int kMultiDefW = 12, kMultiDefK = 4;

// Instances that join the multi-instance launch: gate-by-gate path, points to evaluate, no
// symmetry penalty (its mirrored pre-pass stays with the single call).
bool groupable(const qp_plan* pl, const qp_step_args& a) {
  const int64_t P = a.batch.n_colloc + a.batch.n_ic + a.batch.n_bc;
  return !dense_path(pl) && P > 0 && !(pl->p.w_sym > 0.f);
}

// Signature of a batch's grouped instances: qubits, layers, readout, energy slices and the
// power-of-two bucket of the task count, in order.
uint64_t group_signature(qp_plan* const* plans, const qp_step_args* args, const std::vector<int32_t>& idx) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  for (int32_t i : idx) {
    const qp_plan* pl = plans[i];
    const int ppw = geo_ppw(pl->c.n_qubits);
    const qp_batch& b = args[i].batch;
    const int64_t t = (b.n_colloc + ppw - 1) / ppw + (b.n_ic + ppw - 1) / ppw + (b.n_bc + ppw - 1) / ppw;
    int lg = 0;
    while ((1LL << lg) < t) ++lg;
    mix((uint64_t)pl->c.n_qubits);
    mix((uint64_t)pl->c.n_layers);
    mix((uint64_t)pl->c.n_readout);
    mix((uint64_t)pl->p.energy_nt);
    mix((uint64_t)pl->c.ansatz);
    mix((uint64_t)lg);
  }
  return h;
}

void* multi_kernel_ptr(int n, bool crz) {
  switch (n) {
#define QP_CASE(N) \
  case N: return crz ? (void*)qpk::circuit_multi_kernel<N, true> : (void*)qpk::circuit_multi_kernel<N, false>;
    QP_CASE(1) QP_CASE(2) QP_CASE(3) QP_CASE(4) QP_CASE(5)
    QP_CASE(6) QP_CASE(7) QP_CASE(8) QP_CASE(9) QP_CASE(10)
#undef QP_CASE
  }
  return nullptr;
}

// The grouped instances' loss and gradient: every instance's front launches and argument
// block on stream st[0], one persistent launch per qubit count and QP_MULTI_MAX instances (the
// counts on the streams st[0 .. nst-1] in turn, after an event), then, back on st[0] after the
// launches, every instance's premap backward and reduction over its items.
qp_status launch_grouped(qp_plan* const* plans, const qp_step_args* args, const std::vector<int32_t>& idx,
                         int W, int K, const cudaStream_t* st, int nst, cudaEvent_t fork, const cudaEvent_t* join,
                         int* launches_out) {
  const cudaStream_t s = st[0];
  struct Inst {
    int32_t i;
    WsLayout w;
    const float* pts[3];
    int64_t npts[3];
    QPCircArgs* dst;
    int64_t tpi = 0, items = 0;
  };
  std::vector<Inst> v;
  v.reserve(idx.size());
  int launches = 0;
  int optin = 0;
  for (int32_t i : idx) {
    qp_plan* pl = plans[i];
    const qp_batch* b = &args[i].batch;
    Inst in;
    in.i = i;
    in.pts[0] = b->colloc; in.pts[1] = b->ic; in.pts[2] = b->bc;
    in.npts[0] = b->n_colloc; in.npts[1] = b->n_ic; in.npts[2] = b->n_bc;
    in.w = ws_layout(pl, in.npts[0] + in.npts[1] + in.npts[2]);
    pl->cur_norm[0] = b->norm_colloc; pl->cur_norm[1] = b->norm_ic; pl->cur_norm[2] = b->norm_bc;
    pl->cur_norm_diel = b->norm_colloc > 0 ? b->norm_diel : 0;
    pl->cur_colloc_off = b->colloc_offset;
    pl->last_stream = s;
    pl->last_status = (const int32_t*)((char*)pl->ws + in.w.status);
    const qp_status st = launch_front(pl, args[i].d_params, in.pts, in.npts, in.w, s, true);
    if (st != QP_OK) return st;
    pl->last_launches = front_launches(pl);
    in.dst = (QPCircArgs*)((char*)pl->ws + in.w.desc);
    v.push_back(in);
    if (optin == 0) cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device);
  }
  // argument blocks on st[0]; then one launch per (qubit count, chunk of QP_MULTI_MAX
  // instances), the counts spread over the streams once st[0]'s work so far is done
  struct Launch {
    void* fn;
    int64_t grid;
    int warps, smem;
    qpk::QPMultiArgs ma;
    qp_plan* owner;
  };
  std::vector<Launch> ls;
  for (int g = 0; g < 2 * QP_MAXQ; ++g) {
    const int nq = 1 + g / 2;
    const bool crz = (g & 1) != 0;   // the CRZ-mesh ansatze run in a kernel of their own
    std::vector<int> mem;
    for (int k = 0; k < (int)v.size(); ++k)
      if (plans[v[k].i]->c.n_qubits == nq && qp_has_crz(plans[v[k].i]->c.ansatz) == crz) mem.push_back(k);
    for (size_t c0 = 0; c0 < mem.size(); c0 += QP_MULTI_MAX) {
      const size_t c1 = std::min(mem.size(), c0 + QP_MULTI_MAX);
      // warps per CTA: the largest up to W whose shared-memory layout fits every member
      int Wc = W, smem = 0;
      for (; Wc >= 1; --Wc) {
        smem = 0;
        for (size_t k = c0; k < c1; ++k) {
          const qp_plan* pl = plans[v[mem[k]].i];
          const qpk::SmemLayout lay = qpk::smem_layout(nq, pl->c.n_layers, pl->c.n_readout, pl->p.energy_nt, Wc,
                                                       pl->sstride_grad, geo_ppw(nq), pl->nE, (int)sizeof(QPCircArgs));
          smem = std::max(smem, lay.total);
        }
        if (smem <= optin - 1024) break;   // the kernel's static shared memory (item index)
      }
      if (Wc < 1) return QP_ERR_UNSUPPORTED;
      Launch L;
      std::memset(&L.ma, 0, sizeof(L.ma));
      L.ma.count = (int32_t)(c1 - c0);
      const Inst& f = v[mem[c0]];
      L.owner = plans[f.i];
      L.ma.queue = (unsigned long long*)((char*)plans[f.i]->ws + f.w.status + 192);
      int64_t acc = 0;
      for (size_t k = c0; k < c1; ++k) {
        Inst& in = v[mem[k]];
        qp_plan* pl = plans[in.i];
        QPCircArgs a;
        fill_circ(pl, a, in.w, args[in.i].d_params, in.pts, in.npts, true);
        a.want_dtheta = pl->c.premap == QP_PREMAP_RFF_MLP ? 1 : 0;
        const int64_t tasks = a.task_end[2];
        // at most the plan's partial slots per instance
        const int64_t minp = (tasks + pl->blocks_grad - 1) / pl->blocks_grad;
        in.tpi = std::max<int64_t>((int64_t)Wc * K, minp);
        in.items = (tasks + in.tpi - 1) / in.tpi;
        qpk::store_desc_kernel<<<1, 256, 0, s>>>(a, in.dst, k == c0 ? L.ma.queue : nullptr);
        if (cudaGetLastError() != cudaSuccess) return QP_ERR_CUDA;
        pl->last_launches += 1;
        L.ma.desc[k - c0] = in.dst;
        L.ma.tasks_per_item[k - c0] = (int32_t)in.tpi;
        acc += in.items;
        L.ma.item_end[k - c0] = acc;
      }
      L.fn = multi_kernel_ptr(nq, crz);
      if (raise_smem_limit(L.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return QP_ERR_CUDA;
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L.fn, Wc * 32, smem);
      if (per_sm < 1) per_sm = 1;
      const int64_t cap = (int64_t)plans[f.i]->sm_count * per_sm;
      L.grid = acc < cap ? acc : cap;
      L.warps = Wc;
      L.smem = smem;
      if (L.grid > 0) ls.push_back(L);
    }
  }
  const int ns = std::min<int>(nst, (int)ls.size());
  if (ns > 1) {
    if (cudaEventRecord(fork, s) != cudaSuccess) return QP_ERR_CUDA;
    for (int j = 1; j < ns; ++j)
      if (cudaStreamWaitEvent(st[j], fork, 0) != cudaSuccess) return QP_ERR_CUDA;
  }
  for (size_t k = 0; k < ls.size(); ++k) {
    Launch& L = ls[k];
    void* kargs[] = {&L.ma};
    if (cudaLaunchKernel(L.fn, dim3((unsigned)L.grid), dim3(L.warps * 32), kargs, L.smem, st[k % ns]) != cudaSuccess)
      return QP_ERR_CUDA;
    L.owner->last_launches += 1;
    launches += 1;
  }
  for (int j = 1; j < ns; ++j) {
    if (cudaEventRecord(join[j], st[j]) != cudaSuccess) return QP_ERR_CUDA;
    if (cudaStreamWaitEvent(s, join[j], 0) != cudaSuccess) return QP_ERR_CUDA;
  }
  for (const Inst& in : v) {
    qp_plan* pl = plans[in.i];
    const bool mlp = pl->c.premap == QP_PREMAP_RFF_MLP;
    if (mlp) {
      const qp_status stb = launch_premap_bwd(pl, in.w, args[in.i].d_params, in.pts, in.npts, s);
      if (stb != QP_OK) return stb;
      pl->last_launches += premap_bwd_launches(pl);
    }
    const qp_status str = launch_reduce(pl, in.w, args[in.i].d_params, in.npts, args[in.i].d_loss,
                                        args[in.i].d_grad, mlp, s, 0, in.items);
    if (str != QP_OK) return str;
    pl->last_launches += 1;
  }
  if (launches_out) *launches_out = launches;
  return cuda_status(cudaGetLastError());
}

qp_status check_batch(qp_plan* const* plans, int32_t count, const qp_step_args* args) {
  if (count < 0 || (count > 0 && (!plans || !args))) return QP_ERR_INVALID_ARG;
  for (int32_t i = 0; i < count; ++i) {
    for (int32_t j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return QP_ERR_INVALID_ARG;
    const qp_status c = check_loss_args(plans[i], args[i].d_params, &args[i].batch, args[i].d_loss, args[i].d_grad);
    if (c != QP_OK) return c;
  }
  return QP_OK;
}
}  // namespace

qp_status qp_batch_step_flags(qp_plan* const* plans, int32_t count, const qp_step_args* args, void* stream,
                              uint32_t flags) {
  if (flags & ~(uint32_t)QP_BATCH_NO_GROUPING) return QP_ERR_INVALID_ARG;
  const qp_status chk = check_batch(plans, count, args);
  if (chk != QP_OK) return chk;
  if (count == 0) return QP_OK;
  BatchStreams* bs = batch_streams();
  if (!bs) return QP_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> grouped, rest;
  for (int32_t i = 0; i < count; ++i) {
    if (!(flags & QP_BATCH_NO_GROUPING) && groupable(plans[i], args[i])) grouped.push_back(i);
    else rest.push_back(i);
  }
  // longest first, each onto the least loaded stream (work ~ rows x layers x qubits x 2^n); the
  // grouped instances count as one job on stream 0
  auto cost_of = [&](int32_t i) {
    const qp_batch& b = args[i].batch;
    const qp_circuit& c = plans[i]->c;
    return (double)(4 * b.n_colloc + b.n_ic + b.n_bc + 1) * c.n_layers * c.n_qubits * (double)(1 << c.n_qubits);
  };
  std::vector<int32_t> order(rest);
  std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cost_of(x) > cost_of(y); });
  const int jobs = (int)rest.size() + (grouped.empty() ? 0 : 1);
  const int nst = jobs < QP_BATCH_STREAMS ? jobs : QP_BATCH_STREAMS;
  double load[QP_BATCH_STREAMS] = {0};
  if (cudaEventRecord(bs->fork, s) != cudaSuccess) return QP_ERR_CUDA;
  for (int k = 0; k < nst; ++k)
    if (cudaStreamWaitEvent(bs->st[k], bs->fork, 0) != cudaSuccess) return QP_ERR_CUDA;
  qp_status st = QP_OK;
  if (!grouped.empty()) {
    double gc = 0.0;
    for (int32_t i : grouped) gc += cost_of(i);
    load[0] = gc;
    const qp_plan* p0 = plans[grouped[0]];
    const uint64_t sig = group_signature(plans, args, grouped);
    const bool tuned = p0->mt_sig == sig && p0->mt_warps > 0;
    cudaStream_t gs[QP_GROUP_STREAMS] = {bs->st[0], bs->gst[1], bs->gst[2], bs->gst[3]};
    st = launch_grouped(plans, args, grouped, tuned ? p0->mt_warps : kMultiDefW, tuned ? p0->mt_items : kMultiDefK,
                        gs, QP_GROUP_STREAMS, bs->gfork, bs->gjoin, nullptr);
  }
  for (size_t oi = 0; oi < order.size() && st == QP_OK; ++oi) {
    const int32_t i = order[oi];
    int k = 0;
    for (int q = 1; q < nst; ++q)
      if (load[q] < load[k]) k = q;
    load[k] += cost_of(i);
    st = qp_loss_grad(plans[i], args[i].d_params, &args[i].batch, args[i].d_loss, args[i].d_grad, bs->st[k]);
  }
  for (int k = 0; k < nst; ++k) {
    if (cudaEventRecord(bs->join[k], bs->st[k]) != cudaSuccess) return QP_ERR_CUDA;
    if (cudaStreamWaitEvent(s, bs->join[k], 0) != cudaSuccess) return QP_ERR_CUDA;
  }
  return st;
}

qp_status qp_batch_step(qp_plan* const* plans, int32_t count, const qp_step_args* args, void* stream) {
  return qp_batch_step_flags(plans, count, args, stream, 0u);
}

qp_status qp_batch_tune(qp_plan* const* plans, int32_t count, const qp_step_args* args, void* stream,
                        int32_t* chosen) {
  const qp_status chk = check_batch(plans, count, args);
  if (chk != QP_OK) return chk;
  std::vector<int32_t> grouped;
  for (int32_t i = 0; i < count; ++i)
    if (groupable(plans[i], args[i])) grouped.push_back(i);
  if (grouped.empty()) {
    if (chosen) { chosen[0] = 0; chosen[1] = 0; }
    return QP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  BatchStreams* bs = batch_streams();
  if (!bs) return QP_ERR_CUDA;
  cudaStream_t gs[QP_GROUP_STREAMS] = {s, bs->gst[1], bs->gst[2], bs->gst[3]};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return QP_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return QP_ERR_INVALID_ARG;   // times on the device: not capturable
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QP_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return QP_ERR_CUDA; }
  float best = -1.f;
  int bw = kMultiDefW, bk = kMultiDefK;
  qp_status st = QP_OK;
  for (int wi = 0; wi < 3 && st == QP_OK; ++wi) {
    for (int ki = 0; ki < 3 && st == QP_OK; ++ki) {
      // one warm-up run, then the timed one
      st = launch_grouped(plans, args, grouped, kMultiW[wi], kMultiK[ki], gs, QP_GROUP_STREAMS, bs->gfork,
                          bs->gjoin, nullptr);
      if (st != QP_OK) break;
      if (cudaEventRecord(e0, s) != cudaSuccess) { st = QP_ERR_CUDA; break; }
      st = launch_grouped(plans, args, grouped, kMultiW[wi], kMultiK[ki], gs, QP_GROUP_STREAMS, bs->gfork,
                          bs->gjoin, nullptr);
      if (st != QP_OK) break;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { st = QP_ERR_CUDA; break; }
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { st = QP_ERR_CUDA; break; }
      if (best < 0.f || ms < best) { best = ms; bw = kMultiW[wi]; bk = kMultiK[ki]; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != QP_OK) return st;
  const uint64_t sig = group_signature(plans, args, grouped);
  for (int32_t i : grouped) {
    plans[i]->mt_sig = sig;
    plans[i]->mt_warps = bw;
    plans[i]->mt_items = bk;
  }
  if (chosen) { chosen[0] = bw; chosen[1] = bk; }
  return QP_OK;
}


extern "C" qp_status qp_forward_noalloc(qp_plan* pl, const float* d_params, const float* d_pts,
                                        int64_t B, float* d_fields, float* d_dfields, void* stream) {
  if (!pl || !d_params || B < 0 || (B > 0 && (!d_pts || !d_fields))) return QP_ERR_INVALID_ARG;
  pl->last_launches = 0;
  if (B == 0) return QP_OK;
  const int n = pl->c.n_qubits, L = pl->c.n_layers, ppw = geo_ppw(n);
  // scratch layout: status/counters, gate tables, Pauli coordinates, per-point theta and J
  const size_t off_status = 0;
  const size_t off_gates = al256(off_status + 256);
  const size_t off_cmat = al256(off_gates + (size_t)QP_MAXL * QP_MAXQ * 8 * 4);
  const size_t off_cenc = al256(off_cmat + (size_t)QP_MAXL * QP_MAXQ * 3 * 4 * 4);
  const size_t off_crz = al256(off_cenc + (size_t)QP_MAXQ * 4 * 4);
  const bool crz = qp_has_crz(pl->c.ansatz);
  const size_t off_theta = al256(off_crz + (crz ? (size_t)L * ((size_t)1 << n) * 8 : 0));
  if ((uint64_t)B > (kNoAllocScratchBytes - off_theta) / ((size_t)n * 16)) return QP_ERR_BUFFER_TOO_SMALL;
  if (pl->deep) return QP_ERR_UNSUPPORTED;   // the layer-by-layer premap keeps per-layer rows
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  qp_status st = noalloc_scratch_address(s, &base);
  if (st != QP_OK) return st;
  char* ws = (char*)base;
  pl->last_stream = s;
  pl->last_status = (const int32_t*)(ws + off_status);

  qpk::PrepArgs pa;
  pa.params = d_params; pa.circ_off = pl->circ_off; pa.n = n; pa.L = L;
  pa.ansatz = pl->c.ansatz; pa.enc = pl->c.enc;
  pa.gates = (float*)(ws + off_gates); pa.cmat = (float*)(ws + off_cmat);
  pa.cenc = (float*)(ws + off_cenc);
  pa.counts = (int32_t*)(ws + off_status) + 1;  // zeroed by prep_kernel on every call
  pa.status = (int32_t*)(ws + off_status);
  qpk::prep_kernel<<<(L * n + 63) / 64, 64, 0, s>>>(pa);
  if (crz) {
    const int64_t tot = (int64_t)L << n;
    qpk::crz_phase_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        d_params, pl->circ_off, n, L, pl->c.ansatz, (float2*)(ws + off_crz), nullptr);
  }

  qpk::PremapArgs ma;
  std::memset(&ma, 0, sizeof(ma));
  ma.pts[0] = d_pts; ma.npts[0] = B; ma.ptot = B;
  ma.params = d_params; ma.n = n; ma.premap = pl->c.premap; ma.scale = pl->c.scale;
  ma.n_direct = pl->c.n_direct; ma.F = pl->c.rff_freqs; ma.H = pl->c.mlp_width;
  ma.thetaJ = (float*)(ws + off_theta);
  ma.counts = pa.counts; ma.medium = pl->p.medium; ma.status = pa.status;
  ma.disk_r = pl->p.disk_r; ma.disk_x0 = pl->p.disk_x0; ma.disk_y0 = pl->p.disk_y0;
  const int64_t pb = (B + 127) / 128;
  const int pblocks = (int)(pb < pl->sm_count * 8 ? pb : pl->sm_count * 8);
  if (pl->c.premap == QP_PREMAP_RFF_MLP) {
    void* margs[] = {&ma};
    if (cudaLaunchKernel(premap_fwd_ptr(pl->c.mlp_width), dim3(pblocks), dim3(128), margs,
                         pl->smem_premap, s) != cudaSuccess)
      return QP_ERR_CUDA;
  } else {
    qpk::premap_fwd_kernel<4><<<pblocks, 128, 0, s>>>(ma);
  }

  QPCircArgs a;
  std::memset(&a, 0, sizeof(a));
  a.s = pl->sched;
  fill_problem(pl, a.pb);
  a.n = n; a.L = L; a.m = pl->c.n_readout; a.enc = pl->c.enc;
  a.sstride = pl->sstride_fwd;
  a.pts[0] = d_pts; a.npts[0] = B;
  const int64_t tasks = (B + ppw - 1) / ppw;
  a.task_end[0] = a.task_end[1] = a.task_end[2] = tasks;
  a.thetaJ = (const float*)(ws + off_theta);
  a.gates = (const float*)(ws + off_gates);
  a.crz = crz ? (const float2*)(ws + off_crz) : nullptr;
  a.ansatz = pl->c.ansatz;
  a.nE = pl->nE;
  a.cenc = (const float*)(ws + off_cenc);
  a.head = d_params + pl->head_off;
  a.counts = pa.counts;
  a.want_df = d_dfields != nullptr;
  a.out_f = d_fields;
  a.out_df = d_dfields;
  int64_t blocks = (tasks + pl->warps_fwd - 1) / pl->warps_fwd;
  if (blocks > pl->blocks_fwd) blocks = pl->blocks_fwd;
  void* args[] = {&a};
  if (cudaLaunchKernel(circuit_kernel_ptr(n, false, qp_has_crz(pl->c.ansatz)), dim3((unsigned)blocks), dim3(pl->warps_fwd * 32),
                       args, pl->smem_fwd, s) != cudaSuccess)
    return QP_ERR_CUDA;
  pl->last_launches = crz ? 4 : 3;
  return cuda_status(cudaGetLastError());
}
