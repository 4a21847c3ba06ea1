// qp_sched.cpp -- host planner for the gate passes of the SIMT statevector kernel.
//
// A point's statevectors live in shared memory. A "pass" loads, for every lane, the
// 2^LB amplitudes of one coset of the LB local qubits into registers, applies the
// single-qubit gates of those qubits (Sec. 2.3, Eq. 28) and stores them back.
//
// The CNOTs that end each ansatz layer (a ring, or the all-pairs mesh) are a permutation
// k -> C k of basis indices that is linear over GF(2). It is never executed: the planner
// tracks a frame T (logical index -> storage index) and replaces T by T C^-1, so the next
// passes simply address the permuted amplitudes where they already are. The diagonal CRZ
// mesh is applied by the kernel from the logical indices the planner records for the last
// pass of each layer (klog, jlog).
//
// Storage index s is further swizzled (its low 4 bits replaced by an invertible linear
// mix of all its bits) and every point slot XORs a constant into the low bits, so that the
// 16 lanes of a half-warp touch 16 different 8-byte bank pairs whenever possible. The
// planner searches the swizzle and, pass by pass, the qubit grouping, filler qubits and
// lane basis (any basis of the span of the non-local qubits) with the fewest predicted
// conflicts.
#include <cstring>
#include <vector>

#include "qp_common.h"

namespace {

struct Lin {
  int n;
  uint32_t col[QP_MAXQ];
  uint32_t apply(uint32_t v) const {
    uint32_t r = 0;
    for (int b = 0; b < n; ++b)
      if ((v >> b) & 1u) r ^= col[b];
    return r;
  }
};

int pos(int n, int q) { return n - 1 - q; }

Lin identity(int n) {
  Lin m;
  m.n = n;
  for (int b = 0; b < n; ++b) m.col[b] = 1u << b;
  return m;
}

// Basis-index map of the entangling part of layer l (CNOT ring or mesh; the identity where the
// layer has no CNOT), or its inverse.
uint32_t ring_apply(int n, int ansatz, int l, uint32_t k, bool inverse) {
  return inverse ? qp_ent_unmap(n, ansatz, l, k) : qp_ent_map(n, ansatz, l, k);
}

// Storage -> physical swizzle: phys = s with its low 4 bits replaced by A s_lo ^ B s_hi
// (A invertible), i.e. col[b] is the 4-bit image of storage bit b. Invertible by construction.
struct Swz {
  int n;
  uint32_t col[QP_MAXQ];
  uint32_t operator()(uint32_t s) const {
    if (n < 4) return s;
    uint32_t lo = 0;
    for (int b = 0; b < n; ++b)
      if ((s >> b) & 1u) lo ^= col[b];
    return (s & ~0xFu) | lo;
  }
};

// Incremental GF(2) basis for vectors of up to 16 bits.
struct Basis {
  uint32_t v[16];
  int lead[16];
  int r = 0;
  bool insert(uint32_t x) {
    for (int i = 0; i < r; ++i)
      if ((x >> lead[i]) & 1u) x ^= v[i];
    if (!x) return false;
    int lb = 31 - __builtin_clz(x);
    v[r] = x;
    lead[r] = lb;
    ++r;
    return true;
  }
  bool independent(uint32_t x) const {
    for (int i = 0; i < r; ++i)
      if ((x >> lead[i]) & 1u) x ^= v[i];
    return x != 0;
  }
};

struct PassChoice {
  int ql[8];
  uint32_t w[8];  // lane basis (logical indices), g vectors
  int conflict;
};

// Lane basis for local set ql: a basis of span{e_pos(q) : q not local} whose physical
// images are independent in the low `tbits` bits for the first min(g, tbits) vectors.
PassChoice choose_lanes(int n, int lb, const int* ql, const Lin& T, const Swz& swz) {
  PassChoice pc;
  for (int b = 0; b < lb; ++b) pc.ql[b] = ql[b];
  bool local[QP_MAXQ] = {false};
  for (int b = 0; b < lb; ++b) local[ql[b]] = true;
  int nl[QP_MAXQ];
  int g = 0;
  for (int q = 0; q < n; ++q)
    if (!local[q]) nl[g++] = q;
  const int tbits = g >= 4 ? 4 : g;
  const uint32_t tmask = (1u << tbits) - 1u;
  Basis vecs, imgs;
  int taken = 0;
  for (uint32_t x = 1; x < (1u << g) && taken < tbits; ++x) {
    uint32_t v = 0;
    for (int i = 0; i < g; ++i)
      if ((x >> i) & 1u) v |= 1u << pos(n, nl[i]);
    uint32_t im = swz(T.apply(v)) & tmask;
    if (!vecs.independent(v) || !imgs.independent(im)) continue;
    vecs.insert(v);
    imgs.insert(im);
    pc.w[taken++] = v;
  }
  const int good = taken;
  for (int i = 0; i < g && taken < g; ++i) {
    uint32_t v = 1u << pos(n, nl[i]);
    if (vecs.insert(v)) pc.w[taken++] = v;
  }
  pc.conflict = 1 << (tbits - good);
  return pc;
}

bool invertible4(const uint32_t* c) {
  Basis b;
  for (int i = 0; i < 4; ++i)
    if (!b.insert(c[i])) return false;
  return true;
}

// Plan every pass for one swizzle; returns the summed predicted conflict factor.
int plan_with(int n, int L, int ansatz, const Swz& swz, QPSched* out) {
  const int lb = out->lb, g = n - lb, GL = 1 << g, npl = out->npl;
  Lin T = identity(n);
  int score = 0, worst = 1;
  for (int l = 0; l < L; ++l) {
    bool used[QP_MAXQ] = {false};
    for (int p = 0; p < npl; ++p) {
      const int P = l * npl + p;
      int remaining[QP_MAXQ], nr = 0;
      for (int q = 0; q < n; ++q)
        if (!used[q]) remaining[nr++] = q;
      const int ng = nr < lb ? nr : lb;
      const int nf = lb - ng;
      PassChoice best;
      best.conflict = 1 << 30;
      int best_gates[8] = {0};
      // gate set: ng qubits from the remaining ones; fillers: nf qubits from the rest
      for (uint32_t gm = 0; gm < (1u << nr); ++gm) {
        if (__builtin_popcount(gm) != ng) continue;
        int ql[8], k = 0;
        bool isg[QP_MAXQ] = {false};
        for (int i = 0; i < nr; ++i)
          if ((gm >> i) & 1u) { ql[k++] = remaining[i]; isg[remaining[i]] = true; }
        int others[QP_MAXQ], no = 0;
        for (int q = 0; q < n; ++q)
          if (!isg[q]) others[no++] = q;
        for (uint32_t fm = 0; fm < (1u << no); ++fm) {
          if (__builtin_popcount(fm) != nf) continue;
          int kk = ng;
          for (int i = 0; i < no; ++i)
            if ((fm >> i) & 1u) ql[kk++] = others[i];
          PassChoice pc = choose_lanes(n, lb, ql, T, swz);
          if (pc.conflict < best.conflict) {
            best = pc;
            for (int i = 0; i < ng; ++i) best_gates[i] = ql[i];
          }
          if (best.conflict == 1) break;
        }
        if (best.conflict == 1) break;
      }
      for (int i = 0; i < ng; ++i) used[best_gates[i]] = true;
      score += best.conflict;
      if (best.conflict > worst) worst = best.conflict;
      out->ngate[P] = (uint8_t)ng;
      for (int b = 0; b < lb; ++b) out->ql[P][b] = (uint8_t)best.ql[b];
      for (int lane = 0; lane < 32; ++lane) {
        const int l_in = lane % GL, slot = lane / GL;
        uint32_t K = 0;
        for (int i = 0; i < g; ++i)
          if ((l_in >> i) & 1) K ^= best.w[i];
        uint32_t a = swz(T.apply(K));
        if (g < 4 && n >= 4) a ^= (uint32_t)((slot % (16 / GL)) << g);
        out->lane_addr[P][lane] = (uint16_t)a;
        if (P == 0) out->enc_k[lane] = (uint16_t)K;
        if (p == npl - 1) out->klog[l][lane] = (uint16_t)K;
        if (l == L - 1 && p == npl - 1) {
          uint32_t Ck = ring_apply(n, ansatz, l, K, false);
          uint16_t msk = 0;
          for (int i = 0; i < n; ++i)
            if ((Ck >> pos(n, i)) & 1u) msk |= (uint16_t)(1u << i);
          out->ro_mask[lane] = msk;
        }
      }
      for (int j = 0; j < (1 << lb); ++j) {
        uint32_t sv = 0;
        for (int b = 0; b < lb; ++b)
          if ((j >> b) & 1) sv |= 1u << pos(n, best.ql[b]);
        out->joff[P][j] = (uint16_t)swz(T.apply(sv));
        if (p == npl - 1) out->jlog[l][j] = (uint16_t)sv;
      }
      if (l == L - 1 && p == npl - 1) {
        for (int i = 0; i < n; ++i) {
          uint8_t a = 0;
          for (int b = 0; b < lb; ++b) {
            uint32_t Ce = ring_apply(n, ansatz, l, 1u << pos(n, best.ql[b]), false);
            if ((Ce >> pos(n, i)) & 1u) a |= (uint8_t)(1u << b);
          }
          out->ro_sel[i] = a;
        }
      }
    }
    // frame update: T <- T o C_l^-1
    Lin Tn;
    Tn.n = n;
    for (int b = 0; b < n; ++b) Tn.col[b] = T.apply(ring_apply(n, ansatz, l, 1u << b, true));
    T = Tn;
  }
  out->conflict_max = worst;
  return score;
}

}  // namespace

// Build the pass schedule for n qubits, L layers and an ansatz. Returns 0 on success.
// Tries a few swizzles (a structured one whose low-bit images of any 5 storage bits span
// all 16 bank pairs, then seeded random ones) and keeps the one with the fewest predicted
// bank conflicts; deterministic for a given (n, L, ansatz).
extern "C" int qp_build_sched(int n, int L, int ansatz, QPSched* out) {
  if (n < 1 || n > QP_MAXQ || L < 1 || L > QP_MAXL) return 1;
  const int lb = n <= 3 ? n : (n <= 8 ? 3 : n - 5);
  const int npl = (n + lb - 1) / lb;
  if (L * npl > QP_MAXP) return 2;
  QPSched best, cur;
  int best_score = 1 << 30;
  std::memset(&best, 0, sizeof(best));
  uint32_t rng = 0x9E3779B9u ^ (uint32_t)(n * 131 + L * 17 + ansatz);
  const int ncand = n < 4 ? 1 : 48;
  for (int cand = 0; cand < ncand; ++cand) {
    Swz swz;
    swz.n = n;
    if (cand == 0) {
      // columns: identity on the low bits, odd-weight vectors for the high bits
      static const uint32_t hi[6] = {7, 11, 13, 14, 3, 5};
      for (int b = 0; b < n; ++b) swz.col[b] = b < 4 ? (1u << b) : hi[b - 4];
    } else if (cand == 1) {
      // every column with bit 0 set (useful when one lane bit must land on bit 0)
      static const uint32_t c1[10] = {1, 3, 5, 9, 15, 7, 11, 13, 14, 6};
      for (int b = 0; b < n; ++b) swz.col[b] = c1[b];
      if (!invertible4(swz.col)) continue;
    } else {
      do {
        for (int b = 0; b < n; ++b) {
          rng = rng * 1664525u + 1013904223u;
          swz.col[b] = (rng >> 24) & 0xFu;
        }
      } while (n >= 4 && !invertible4(swz.col));
    }
    std::memset(&cur, 0, sizeof(cur));
    cur.npl = npl;
    cur.npass = L * npl;
    cur.lb = lb;
    const int score = plan_with(n, L, ansatz, swz, &cur);
    if (score < best_score) {
      best_score = score;
      best = cur;
    }
    if (best_score == L * npl) break;
  }
  *out = best;
  return 0;
}
