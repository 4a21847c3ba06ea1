// qp_common.h -- definitions shared by the host planner, the C-ABI and the kernels.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#define QP_MAXQ 10      // qubits
#define QP_MAXL 16      // ansatz layers
#define QP_MAXP 48      // gate passes (layers x passes per layer)
#define QP_MAXNT 256    // energy slices
#define QP_NLP 7        // loss partial sums: res1 vac, res1 diel, res2, res3, energy, ic, bc
#define QP_NLOSS_OUT 9  // loss terms written before the energy slices (QP_NLOSS of qpinn.h)
#define QP_MAXF 256     // RFF frequencies
#define QP_MAXH 64      // MLP width of the fused one-hidden-layer premap kernels

// Geometry of one statevector per point group (compile-time per qubit count).
//   LB   : qubits held in registers per lane ("local" qubits of a pass)
//   GL   : lanes that share one point (2^(n-LB))
//   PPW  : points per warp
template <int NQ>
struct QPGeo {
  static constexpr int LB = NQ <= 3 ? NQ : (NQ <= 8 ? 3 : NQ - 5);
  static constexpr int AMPS = 1 << LB;
  static constexpr int GL = 1 << (NQ - LB);
  static constexpr int PPW = 32 / GL;
  static constexpr int DIM = 1 << NQ;
};

// Pass schedule produced on the host (see qp_sched.cpp). Pass P = l * npl + p applies the
// single-qubit gates of layer l to the qubits ql[P][0 .. ngate[P]-1]; lane `lane` holds,
// for register j, the amplitude stored at shared-memory index lane_addr[P][lane] ^ joff[P][j]
// of each vector of its point (float2 units).
struct QPSched {
  int32_t npass, npl, lb;
  uint8_t ngate[QP_MAXP];
  uint8_t ql[QP_MAXP][8];
  uint16_t lane_addr[QP_MAXP][32];
  uint16_t joff[QP_MAXP][32];
  uint16_t enc_k[32];    // logical basis index of each lane's register 0 in pass 0 (frame = I)
  uint16_t ro_mask[32];  // readout: bit i set -> lane's sign for Z_i flips
  uint8_t ro_sel[16];    // readout: Walsh index (over local bits) of Z_i in the last pass
  int32_t conflict_max;  // planner's worst predicted bank-conflict factor
  // last pass of each layer (CRZ mesh ansatze: no CNOT, so the frame stays the identity):
  // logical basis index of each lane's register 0, and of register j relative to it
  uint16_t klog[QP_MAXL][32];
  uint16_t jlog[QP_MAXL][32];
};

// Ansatz properties shared by the host and the kernels (qp_ansatz of qpinn.h).
__host__ __device__ inline bool qp_has_crz(int ansatz) { return ansatz == 4 || ansatz == 5; }
// single-qubit angles per qubit and layer: RY, RZ (0); RX (4); RX, RZ (5); Rot (1, 2, 3, 6)
__host__ __device__ inline int qp_ansatz_k(int ansatz) {
  return ansatz == 0 || ansatz == 5 ? 2 : (ansatz == 4 ? 1 : 3);
}
// circuit parameters per layer: single-qubit angles, then n (n-1) CRZ angles [i][j != i]
__host__ __device__ inline int qp_layer_params(int ansatz, int n) {
  return n * qp_ansatz_k(ansatz) + (qp_has_crz(ansatz) ? n * (n - 1) : 0);
}
// CRZ gradient sums per layer: Z_t for every qubit t, then Z_ct for every pair c < t
__host__ __device__ inline int qp_crz_sums(int ansatz, int n) {
  return qp_has_crz(ansatz) ? n + n * (n - 1) / 2 : 0;
}
// index of the pair (c, t), c < t, among the pairs of n qubits
__host__ __device__ inline int qp_pair_index(int n, int c, int t) { return c * (2 * n - c - 1) / 2 + (t - c - 1); }
// Entangling permutation of layer l on basis index k (CNOT ring or CNOT mesh; identity for
// the no-entanglement and CRZ ansatze, whose mesh is diagonal). Qubit q is bit n-1-q.
__host__ __device__ inline uint32_t qp_ent_map(int n, int ansatz, int l, uint32_t k) {
  if (n < 2 || ansatz == 3 || ansatz == 4 || ansatz == 5) return k;
  if (ansatz == 6) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (j != i && ((k >> (n - 1 - i)) & 1u)) k ^= 1u << (n - 1 - j);
    return k;
  }
  const int r = ansatz == 2 ? 1 + (l % (n - 1)) : 1;
  for (int i = 0; i < n; ++i)
    if ((k >> (n - 1 - i)) & 1u) k ^= 1u << (n - 1 - (i + r) % n);
  return k;
}
// Its inverse (the gates in reverse order).
__host__ __device__ inline uint32_t qp_ent_unmap(int n, int ansatz, int l, uint32_t k) {
  if (n < 2 || ansatz == 3 || ansatz == 4 || ansatz == 5) return k;
  if (ansatz == 6) {
    for (int i = n - 1; i >= 0; --i)
      for (int j = n - 1; j >= 0; --j)
        if (j != i && ((k >> (n - 1 - i)) & 1u)) k ^= 1u << (n - 1 - j);
    return k;
  }
  const int r = ansatz == 2 ? 1 + (l % (n - 1)) : 1;
  for (int i = n - 1; i >= 0; --i)
    if ((k >> (n - 1 - i)) & 1u) k ^= 1u << (n - 1 - (i + r) % n);
  return k;
}

struct QPProblemDev {
  int32_t medium;
  float eps_r, disk_r, disk_x0, disk_y0, sigmoid_w;
  float ic_sigma, ic_x0, ic_y0, w_ic, w_bc, w_energy;
  int32_t energy_slice, energy_nt;
  int32_t phys_loss;   // 0: Eq. 13, 1: Eqs. 34-35 (dielectric case)
  float w_sym;         // weight of L_sym (Eq. 18), 0 = off
  // sharding of one loss over several calls: whole-loss counts of the collocation, IC and BC
  // sets (0: this call's), whole-set points inside the disk (read when norm[0] > 0), global
  // index of this call's first collocation point (energy slices)
  int64_t norm[3], norm_diel, colloc_off;
};

// Arguments of the circuit kernel (passed by value; the schedule is copied to shared memory).
struct QPCircArgs {
  QPSched s;
  QPProblemDev pb;
  int32_t n, L, m, enc;
  int32_t sstride;            // float2 per point slot in shared memory
  int32_t want_dtheta;        // write per-point dL/dtheta, dL/dJ
  int32_t want_df;            // forward mode: derivatives requested
  const float* pts[3];        // colloc, ic, bc
  int64_t npts[3];
  int64_t task_end[3];        // cumulative warp-task counts per set
  int64_t pt_base[3];         // first global point index of each set (theta/J rows)
  const float* thetaJ;        // [P][n][4] (theta, dtheta/dx, dtheta/dy, dtheta/dt)
  float* dthetaJ;             // [P][n][4] (dL/dtheta, dL/dJ_x, dL/dJ_y, dL/dJ_t)
  const float* gates;         // [L][n][8] forward 2x2 complex gate per qubit and layer
  const float2* crz;          // CRZ mesh ansatze: [L][2^n] phase (cos, sin) by logical index
  int32_t ansatz;
  int32_t nE;                 // gate-gradient partial sums per block (3 n L + L crz sums)
  const float* cenc;          // [n][4] Pauli coefficients of the embedding generator
  const float* head;          // W[3][m], b[3]
  const int32_t* counts;      // [0] dielectric-set size
  double* blk_loss;           // [grid][QP_NLP + nt]
  float* blk_grad;            // [grid][3 n L + 3 m + 3]
  float* out_f;               // forward mode [B][3] (all sets, by global point index)
  float* out_df;              // forward mode [B][3][3]
  int32_t loss_stride, grad_stride;
  // symmetry penalty (Eq. 18): extra cotangents of the collocation points' fields, and the rows
  // of set 2 from index nbc on (the mirrored points) whose cotangents are given, not a loss's
  const float* gsym;          // [n colloc][3] or null
  const float* gext;          // [npts[2] - nbc][3] or null
  int64_t nbc;                // boundary points of set 2 (the rest are the given-cotangent rows)
};
