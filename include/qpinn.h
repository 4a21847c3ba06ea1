/* qpinn.h -- C-ABI of the B300 QPINN hot-path library (libqpinn.so).
 *
 * The library evaluates the hybrid quantum PINN of arxiv 2506.23246 at a batch of
 * collocation points on one GPU: premap (direct angle map, or random Fourier
 * features + tanh MLP, Sec. 2.2), angle embedding and ansatz layers of the
 * parametrized quantum circuit (Sec. 2.3, Eqs. 27-28), Pauli-Z readout and a linear
 * head to the fields (Ez, Hx, Hy); exact first derivatives d/dx, d/dy, d/dt by
 * forward-mode tangent states; the 2D TM Maxwell residuals and losses (Eqs. 8-17),
 * the Poynting energy residual (Eq. 23), the total loss (Eq. 24), the energy slice
 * sums U(t) (Eq. 31); and gradients of the total loss with respect to every
 * parameter by a reverse (adjoint) sweep through the tangent states.
 *
 * Conventions shared by every call:
 *  - All arrays are row-major and contiguous. Points are float32 [B][3] = (x, y, t).
 *  - Pointers named d_* are device pointers owned by the caller. The library never
 *    allocates device memory in a compute call and never synchronises the stream
 *    (except qp_last_device_error). Scratch comes from a caller-owned workspace set
 *    with qp_set_workspace.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Gates use the half-angle convention RX(t) = exp(-i t X / 2) (so <Z> = cos t after
 *    RX(t) on |0>, Fig. 3); Rot(a, b, g) = RZ(g) RY(b) RZ(a) (Eq. 28); qubit q is bit
 *    (n-1-q) of the basis index; the CNOT ring of layer l is CNOT(i, (i+r) mod n) for
 *    i = 0..n-1 in order, r = 1 (Basic) or 1 + (l mod (n-1)) (Strongly entangling).
 *  - Every call returns a qp_status; argument errors are detected on the host before
 *    any launch; no C++ exception crosses this boundary.
 */
#ifndef QPINN_H
#define QPINN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QP_OK = 0,
  QP_ERR_INVALID_ARG = 1,      /* null pointer, bad enum value, inconsistent sizes */
  QP_ERR_UNSUPPORTED = 2,      /* valid request outside what this library implements */
  QP_ERR_BUFFER_TOO_SMALL = 3, /* workspace missing or smaller than qp_workspace_size */
  QP_ERR_CUDA = 4,             /* a CUDA runtime call failed (launch error, bad device) */
  QP_ERR_NONFINITE = 5,        /* the device saw a non-finite loss (reported via status) */
  QP_ERR_TIMEOUT = 6,          /* a bounded device-side wait ran out */
  QP_ERR_INTERNAL = 7
} qp_status;

/* Ansatz layers (Sec. 2.3). Each layer applies one single-qubit gate per qubit, then its
 * entangling part:
 *   BASIC_RYRZ       RY(a) then RZ(b); CNOT ring of stride 1
 *   BASIC_ROT        Rot(a, b, g) (Eq. 28); CNOT ring of stride 1
 *   STRONG_ROT       Rot; CNOT ring of stride 1 + (l mod (n-1))
 *   NOENT_ROT        Rot; no two-qubit gate
 *   CROSS_MESH       RX(a); CRZ(i, j) for every ordered pair i != j, each with its own angle
 *                    (Eq. 29; control i, target j, CRZ(t) = RZ(t) on j where qubit i is 1)
 *   CROSS_MESH_2ROT  RX(a) then RZ(b); the same CRZ mesh
 *   CROSS_MESH_CNOT  Rot; CNOT(i, j) for every ordered pair i != j
 * The mesh gates run i = 0..n-1 (outer) and j = 0..n-1, j != i (inner), in that order. */
typedef enum {
  QP_ANSATZ_BASIC_RYRZ = 0,
  QP_ANSATZ_BASIC_ROT = 1,
  QP_ANSATZ_STRONG_ROT = 2,
  QP_ANSATZ_NOENT_ROT = 3,
  QP_ANSATZ_CROSS_MESH = 4,
  QP_ANSATZ_CROSS_MESH_2ROT = 5,
  QP_ANSATZ_CROSS_MESH_CNOT = 6
} qp_ansatz;

typedef enum { QP_ENC_RX = 0, QP_ENC_RY = 1 } qp_enc_gate;

/* Angle scalings of Eq. 27a-e: none a, pi a, (a+1) pi/2, asin(a)+pi/2, acos(a). */
typedef enum {
  QP_SCALE_NONE = 0,
  QP_SCALE_PI = 1,
  QP_SCALE_BIAS = 2,
  QP_SCALE_ASIN = 3,
  QP_SCALE_ACOS = 4
} qp_scale;

/* DIRECT: theta_j = scale(v_j) for j < n_direct (v = (x,y,t)), theta_j = 0 otherwise.
 * RFF_MLP: r = [cos(Omega v), sin(Omega v)] (Sec. 2.2, RFF), mlp_depth tanh layers of
 * width mlp_width, a linear layer to n_qubits, a = tanh(.), theta = scale(a). */
typedef enum { QP_PREMAP_DIRECT = 0, QP_PREMAP_RFF_MLP = 1 } qp_premap;

/* SIMT_FP32: gate-by-gate statevectors in registers and shared memory, FP32 (any n).
 * GEMM_SPLIT: the ansatz layers fused into one 2^n x 2^n unitary applied to all points as
 * tensor-core contractions (tcgen05) on split operands hi + lo with FP32 accumulation, about
 * 22-bit operands: FP16 pairs scaled by powers of two (three FP16 products per term, the hi*hi
 * products and the hi*lo + lo*hi corrections in separate accumulators; the default and the
 * only form of the n = 7, 8 loss kernels) or 3xTF32 (qp_plan_set_operands). Forward for
 * n >= 5, loss + gradient for n >= 7. AUTO picks GEMM_SPLIT for 7-10 qubits, SIMT otherwise.
 * GEMM_BF16X3 is reserved (QP_ERR_UNSUPPORTED): FP16 pairs with power-of-two scaling give
 * the same operand precision with three products instead of six. */
typedef enum {
  QP_PATH_AUTO = 0,
  QP_PATH_SIMT_FP32 = 1,
  QP_PATH_GEMM_SPLIT = 2,
  QP_PATH_GEMM_BF16X3 = 3
} qp_path;

typedef enum { QP_MEDIUM_VACUUM = 0, QP_MEDIUM_DIELECTRIC = 1 } qp_medium;

typedef struct {
  int32_t n_qubits;  /* 1..10 */
  int32_t n_layers;  /* 1..16 */
  int32_t n_readout; /* readout qubits 0..m-1, 1 <= m <= n_qubits */
  int32_t ansatz;    /* qp_ansatz */
  int32_t enc;       /* qp_enc_gate */
  int32_t scale;     /* qp_scale */
  int32_t premap;    /* qp_premap */
  int32_t n_direct;  /* DIRECT premap: inputs mapped to qubits 0..n_direct-1 (<= 3) */
  int32_t rff_freqs; /* RFF_MLP: number of frequencies F (Omega is [F][3]), 1..256 */
  int32_t mlp_width; /* RFF_MLP: hidden width H, 1..1024 */
  int32_t mlp_depth; /* RFF_MLP: number of hidden tanh layers, 0..8 */
  int32_t periodic;  /* RFF_MLP: 1 = the periodic input map of Eqs. 25-26 before the RFF layer,
                        (x, y, t) -> (sin(pi x), cos(pi x), sin(pi y), cos(pi y), sin(2 pi t / T),
                        cos(2 pi t / T)) for the domain lengths 2 of [-1, 1]^2 and a learned time
                        period T; Omega is then [F][6] */
} qp_circuit;

typedef struct {
  int32_t medium;    /* qp_medium */
  float eps_r;       /* dielectric: eps = 1 + (eps_r-1) sigmoid((disk_r - r)/sigmoid_w) */
  float disk_r, disk_x0, disk_y0, sigmoid_w;
  float ic_sigma;    /* initial pulse exp(-((x-ic_x0)^2+(y-ic_y0)^2)/(2 sigma^2)), Eq. 14 */
  float ic_x0, ic_y0;
  float w_ic, w_bc, w_energy; /* loss weights (Eq. 24 uses 10) */
  int32_t energy_slice;       /* collocation point p belongs to energy slice p/energy_slice */
  int32_t energy_nt;          /* number of energy slices U(t_k) reported (0 = none) */
  int32_t phys_loss;          /* dielectric physics loss: 0 Eq. 13 (separate MSEs of res1 over the
                                 vacuum and dielectric sets, 1/eps(x,y) pointwise), 1 the intuitive
                                 form of Eqs. 34-35 (one MSE over all collocation points, eps = 1 or
                                 eps_r by set) */
  float w_sym;                /* weight of the symmetry penalty L_sym (Eq. 18; Eq. 24 uses 10), 0 = off */
} qp_problem;

/* Point sets of one loss evaluation (device pointers, float32 [n][3]). colloc points
 * carry the residual and energy terms; ic points the initial-condition misfit (Eq. 17);
 * bc points the PEC boundary term Ez = 0. Any set may be empty (NULL, 0).
 *
 * Sharding (data parallelism over ranks): the loss terms are means over whole point sets
 * (Eqs. 11-17, 23). When one loss is split over several calls, give each call the whole-loss
 * counts in norm_colloc / norm_ic / norm_bc (each >= this call's count), the whole collocation
 * set's number of points inside the dielectric disk in norm_diel (0 <= norm_diel <=
 * norm_colloc; see qp_count_dielectric; read when norm_colloc > 0) and the global index of
 * this call's first collocation point in colloc_offset (energy slices of Eq. 31; requires
 * colloc_offset + n_colloc <= norm_colloc). The loss terms and gradients of the calls then sum
 * to those of the whole loss. All zero: the call's own sets are the whole loss. Invalid
 * combinations fail with QP_ERR_INVALID_ARG before any launch. */
typedef struct {
  const float* colloc;
  int64_t n_colloc;
  const float* ic;
  int64_t n_ic;
  const float* bc;
  int64_t n_bc;
  int64_t norm_colloc, norm_ic, norm_bc, norm_diel, colloc_offset;
} qp_batch;

/* Layout of d_loss written by qp_loss_grad (float64):
 *  [0] total loss (Eq. 24 without L_sym), [1] L_phys (Eq. 11 or 13), [2] w_ic * L_IC,
 *  [3] w_bc * L_BC, [4] w_energy * mean(Eq. 23 residual^2), [5] MSE(res1) over the vacuum
 *  set (all points in vacuum), [6] MSE(res1) over the dielectric set, [7] MSE(res2),
 *  [8] MSE(res3), [9 .. 9+energy_nt) energy slice sums U(t_k) (Eq. 31), and when w_sym > 0
 *  [9+energy_nt] w_sym * L_sym (Eq. 18: fields at (-x, y, t) and (x, -y, t) of every
 *  collocation point, the x-mirror terms left out in the dielectric case), which the total
 *  [0] includes. Both paths evaluate it: a fields-only pass over the collocation points and
 *  their mirrors gives each mirrored point's field cotangents, and the main pass carries the
 *  mirrored points as extra rows with those cotangents. */
#define QP_NLOSS 9

typedef struct qp_plan qp_plan;

/* Create a plan for one circuit + problem. Host-only: validates the configuration and
 * builds the shared-memory schedule of the gate passes. *out receives the plan (owned
 * by the caller, free with qp_plan_destroy). Fails with QP_ERR_INVALID_ARG for bad
 * values and QP_ERR_UNSUPPORTED for valid ones this library does not implement. */
qp_status qp_plan_create(const qp_circuit* circuit, const qp_problem* problem, int32_t path,
                         qp_plan** out);
void qp_plan_destroy(qp_plan* plan);

/* Number of float32 entries of the flat parameter vector. Layout (Sec. 2.2-2.3):
 *   RFF_MLP premap: Omega[F][3] (Omega[F][6] with the periodic map; fixed, gradient 0), the
 *   learned period T (periodic map only), then per hidden layer W[H][in] (in = 2F first, H
 *   after) and b[H], then W_out[n][H], b_out[n];
 *   circuit, per layer: [n][k] single-qubit angles with k = 2 (RY, RZ) for BASIC_RYRZ, 1 (RX)
 *   for CROSS_MESH, 2 (RX, RZ) for CROSS_MESH_2ROT, else 3 (Rot a, b, g); then, for CROSS_MESH
 *   and CROSS_MESH_2ROT, the n (n-1) CRZ angles [i][j != i] (targets j in increasing order);
 *   head: W[3][m], b[3]. */
qp_status qp_param_count(const qp_plan* plan, int64_t* n_params);
/* offsets[0] circuit block, [1] head block, [2] total, [3] number of fixed (Omega) entries. */
qp_status qp_param_layout(const qp_plan* plan, int64_t* offsets4);

/* Device scratch needed by calls on up to max_points points in total (all sets). */
qp_status qp_workspace_size(const qp_plan* plan, int64_t max_points, size_t* bytes);
/* Attach caller-owned device scratch (>= qp_workspace_size, 256-byte aligned). The
 * plan keeps the pointer; the caller keeps ownership and must not free it while the
 * plan is used. Calls on one plan must not overlap on the GPU (they share it). */
qp_status qp_set_workspace(qp_plan* plan, void* d_workspace, size_t bytes);

/* Fields and input derivatives at B points: d_fields [B][3] = (Ez, Hx, Hy),
 * d_dfields [B][3][3] = d field_c / d (x, y, t)_d, or NULL to skip derivatives. */
qp_status qp_forward(qp_plan* plan, const float* d_params, const float* d_pts, int64_t B,
                     float* d_fields, float* d_dfields, void* stream);

/* Loss terms (layout above, float64 [QP_NLOSS + energy_nt], one more with L_sym) and the gradient of the
 * total loss w.r.t. every parameter (float32 [n_params]; Omega entries get 0). */
qp_status qp_loss_grad(qp_plan* plan, const float* d_params, const qp_batch* batch,
                       double* d_loss, float* d_grad, void* stream);

/* Number of points of d_pts [n][3] strictly inside the problem's dielectric disk (the test the
 * loss uses), written to the device int64 *d_count (overwritten). For sharded losses: the
 * ranks all-reduce their counts into qp_batch.norm_diel. QP_ERR_INVALID_ARG for bad pointers
 * or n < 0; a vacuum problem writes 0. */
qp_status qp_count_dielectric(qp_plan* plan, const float* d_pts, int64_t n, int64_t* d_count,
                              void* stream);

/* Black-hole collapse indicator (Sec. 5, "Black hole" loss landscape) from the energy slices
 * U(t_k) that qp_loss_grad writes into its loss terms ([QP_NLOSS .. QP_NLOSS + energy_nt),
 * float64), on the uniform slice times t_k = t_max k / (energy_nt - 1): the normalised
 * energies U~(t_k) = U(t_k) / U(0) and I_BH = 1 - min over t_k >= delta of U~(t_k) (close to 1:
 * the fields collapsed to the trivial solution after t = 0). d_out: float64 [energy_nt + 1],
 * U~(t_0 .. t_{nt-1}) then I_BH. Device pointers, stream-ordered, no allocation. Not finite
 * when U(0) is not positive. QP_ERR_INVALID_ARG for null pointers, energy_nt < 2 or above
 * the energy-slice limit, t_max <= 0 or delta outside [0, t_max]. */
qp_status qp_bh_indicator(const double* d_loss_terms, int32_t energy_nt, double t_max, double delta,
                          double* d_out, void* stream);

/* One loss evaluation of a batched step (qp_batch_step): parameters, point sets and
 * outputs of one instance, with the meaning they have in qp_loss_grad. */
typedef struct {
  const float* d_params;
  qp_batch batch;
  double* d_loss;
  float* d_grad;
} qp_step_args;

/* Loss and gradient of `count` independent instances (the paper's experiments train many
 * configurations; each instance is its own circuit, problem and point sets) in one call:
 * instance i is qp_loss_grad(plans[i], args[i]...). No counterpart in the paper, which trains
 * one configuration per run; the uneven multi-configuration workload is a throughput target
 * of this library.
 *
 * Instances on the gate-by-gate path (QP_PATH_SIMT_FP32, points to evaluate, no symmetry
 * penalty) share one persistent statevector launch per qubit range (1-7 and 8-10 qubits, up
 * to 64 instances each): every instance's premap and argument block first, then CTAs take
 * items of consecutive warp-tasks (point groups) of any instance from one atomic counter, with
 * the warps per CTA and the tasks per item that qp_batch_tune chose for this mix (12 warps and
 * 4 tasks per warp until then), then every instance's premap backward and reduction. Each
 * item writes its own partial slot, so an instance's loss and gradient are summed over its
 * items (values equal to qp_loss_grad's up to FP32 summation order). The other instances
 * (tensor-core path, symmetry penalty, empty) run as ordinary qp_loss_grad calls. The grouped
 * work and those calls run concurrently on library-owned streams forked from `stream` (the
 * longest call first, each on the least loaded stream) and joined back into it, so work
 * issued on `stream` after the call sees every result; the call is capturable into a CUDA
 * graph on `stream`. Every plan must have its own workspace (the same plan may not appear
 * twice). All arguments are checked before any launch (QP_ERR_INVALID_ARG,
 * QP_ERR_BUFFER_TOO_SMALL, QP_ERR_UNSUPPORTED as qp_loss_grad); the first launch that fails
 * stops the call with its status, after the streams are joined. */
qp_status qp_batch_step(qp_plan* const* plans, int32_t count, const qp_step_args* args, void* stream);

/* qp_batch_step with flags: QP_BATCH_NO_GROUPING runs every instance as its own qp_loss_grad
 * call on the worker streams (no multi-instance launch). Other bits: QP_ERR_INVALID_ARG. */
typedef enum { QP_BATCH_NO_GROUPING = 1 } qp_batch_flags;
qp_status qp_batch_step_flags(qp_plan* const* plans, int32_t count, const qp_step_args* args, void* stream,
                              uint32_t flags);

/* Tuner of the multi-instance launch: runs the grouped instances of this batch (as
 * qp_batch_step would group them) once untimed and once timed with CUDA events on `stream` for
 * every candidate shape (4, 8 or 12 warps per CTA x 1, 4 or 16 warp-tasks per warp and item),
 * and stores the fastest in every grouped plan, keyed by the mix's signature (qubits, layers,
 * readout, energy slices, ansatz and the power-of-two bucket of each instance's task count, in
 * order); qp_batch_step uses it while the signature matches. The outputs in `args` are
 * overwritten with this batch's results. Synchronises `stream`; QP_ERR_INVALID_ARG while the
 * stream is capturing. chosen (may be NULL): [0] warps per CTA, [1] tasks per warp and item
 * (0, 0 when no instance is grouped). */
qp_status qp_batch_tune(qp_plan* const* plans, int32_t count, const qp_step_args* args, void* stream,
                        int32_t* chosen);

/* Synchronise the stream of the last compute call on this plan and return that call's device
 * status word (QP_OK, QP_ERR_NONFINITE or QP_ERR_TIMEOUT; QP_OK before the first call) or
 * QP_ERR_CUDA for a sticky CUDA error. After qp_forward_noalloc the word is the one in the
 * library's fixed array, which the next qp_forward_noalloc call on any plan overwrites. */
qp_status qp_last_device_error(qp_plan* plan);

const char* qp_status_str(qp_status s);

/* Kernel launches issued by the last compute call on this plan (for accounting). */
int32_t qp_last_launch_count(const qp_plan* plan);

/* The path a plan resolved to (QP_PATH_SIMT_FP32 or QP_PATH_GEMM_SPLIT). */
int32_t qp_plan_path(const qp_plan* plan);

/* Operand form of the tensor-core contractions that have two: the forward of qp_forward for
 * n >= 7, and the forward, the weight gradient and the back-projection mu = Re(U'^H lambda)
 * of qp_loss_grad for n = 9, 10 (the n = 7, 8 kernels of qp_loss_grad have FP16 pairs
 * only). FP16_PAIRS (the default): FP16 hi + lo of
 * power-of-two-scaled operands, the hi*hi products and the hi*lo + lo*hi corrections in
 * separate FP32 accumulators. TF32_PAIRS: 3xTF32 in one accumulator. Both are ~22-bit
 * operands; the FP16 form halves the tensor-core time, and the tensor core's truncating
 * accumulation (about one FP32 ulp per instruction) touches the result K/16 times instead
 * of 3K/8.
 * Returns QP_ERR_INVALID_ARG for another value. Not thread-safe against concurrent calls on
 * the same plan. */
typedef enum { QP_OPERANDS_FP16_PAIRS = 0, QP_OPERANDS_TF32_PAIRS = 1 } qp_operands;
qp_status qp_plan_set_operands(qp_plan* plan, int32_t operands);

/* Failure detection, for tests: every wait of the fused forward kernel's pipeline (the
 * tensor-core loss path at n = 7, 8) gives up after `polls` polls of its mbarrier instead of
 * the built-in bound (0 restores it). A wait that runs out stops the kernel cleanly: the waits
 * that let its in-flight copies and MMAs finish keep the built-in bound, tensor memory is freed,
 * and the call's status word reads QP_ERR_TIMEOUT (qp_last_device_error). The plan stays
 * usable; the call's outputs are not meaningful. QP_ERR_INVALID_ARG for a null plan. */
qp_status qp_set_wait_limit(qp_plan* plan, uint32_t polls);

/* Optional profiling: two cudaEvent_t (passed as void*, created by the caller) that the
 * following compute calls record on their stream immediately before and after one measured
 * kernel, so its device time can be read with cudaEventElapsedTime. kernel selects it:
 *   QP_PROF_MAIN (0): the statevector kernel on the SIMT path; on the tensor-core path the
 *     forward contraction (the fused forward kernel of qp_loss_grad for n = 7, 8; the forward
 *     launches of every point set otherwise, and of qp_forward);
 *   QP_PROF_WGRAD (1): the weight-gradient contraction of qp_loss_grad (tensor-core path);
 *   QP_PROF_MU (2): the back-projection mu = Re(U'^H lambda) of qp_loss_grad (tensor-core
 *     path with the RFF + MLP premap; with its embedding-gradient epilogue for n = 7, 8).
 * Pass NULL, NULL to stop. The plan does not own the events. QP_ERR_INVALID_ARG for another
 * kernel value or only one null event. */
typedef enum { QP_PROF_MAIN = 0, QP_PROF_WGRAD = 1, QP_PROF_MU = 2 } qp_prof_kernel;
qp_status qp_set_profile_events(qp_plan* plan, int32_t kernel, void* ev_start, void* ev_stop);

/* Fields and input derivatives like qp_forward, for callers that cannot allocate device memory:
 * code running inside a memory pool that refuses new allocations, a plugin handed a fixed
 * device budget, a host that forbids cudaMalloc after start-up. The paper has no counterpart:
 * this is a library convenience. Instead of the plan's workspace, the call uses one fixed
 * 16 MiB array of device memory owned by the library; every GPU that loads the library keeps
 * that array until the process exits. Nothing is allocated or freed by this call.
 * It always runs the FP32 SIMT path (premap kernel without tensor cores, gate-by-gate circuit
 * kernel), whatever path and operand form the plan names: on a plan with the direct premap and
 * the SIMT path its results equal qp_forward's bit for bit; otherwise both agree with the FP64
 * oracle within the library's 1e-5 relative bar. Plans whose RFF + MLP premap is not one hidden
 * layer of width 4, 8, 16, 32 or 64 are refused with QP_ERR_UNSUPPORTED (their premap keeps
 * every layer's rows for all points).
 * Limit: B * n_qubits * 16 bytes plus about 13 KiB of tables (and L * 2^n * 8 bytes of the CRZ
 * mesh diagonal for the Cross-Mesh ansatze) must fit in 16 MiB (B <= 104,000 points at 10
 * qubits, 130,000 at 8); a larger B is rejected with QP_ERR_BUFFER_TOO_SMALL
 * before anything is launched. The array's device address is looked up with the device current
 * on every call made outside stream capture; a call made while its stream is capturing reuses
 * the address of the last call outside capture on that device, so make one call before any
 * capture (otherwise QP_ERR_CUDA). All calls share the one array and each call overwrites it,
 * so calls that overlap on the GPU (other streams, other plans, other threads) race; serialise
 * them. qp_last_device_error then reads the status word in that array. Arguments, layouts and
 * the other errors are those of qp_forward. */
qp_status qp_forward_noalloc(qp_plan* plan, const float* d_params, const float* d_pts, int64_t B,
                             float* d_fields, float* d_dfields, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QPINN_H */
