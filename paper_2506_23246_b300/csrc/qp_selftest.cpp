// qp_selftest.cpp -- host-only check of the pass schedule.
//
// Emulates, lane by lane, what the circuit kernel does with the planner's tables: the fused
// embedding in pass 0, load / gate / store through lane_addr ^ joff, CNOTs (ring or mesh)
// folded into the frame, a diagonal phase per layer (the CRZ mesh ansatze) applied in the
// layer's last pass by the logical indices klog ^ jlog, and the readout through ro_mask /
// ro_sel with the Walsh transform. The result is compared with a direct gate-by-gate
// simulation that applies every CNOT and every phase explicitly.
// Also checks that every pass touches each amplitude of a point exactly once.
#include <cmath>
#include <complex>
#include <cstdint>
#include <random>
#include <vector>

#include "qp_common.h"

extern "C" int qp_build_sched(int n, int L, int ansatz, QPSched* out);

namespace {
typedef std::complex<double> cd;
struct U2 { cd a, b, c, d; };

void apply_direct(std::vector<cd>& s, int n, int q, const U2& u) {
  const int bit = 1 << (n - 1 - q);
  for (int k = 0; k < (1 << n); ++k) {
    if (k & bit) continue;
    cd x = s[k], y = s[k | bit];
    s[k] = u.a * x + u.b * y;
    s[k | bit] = u.c * x + u.d * y;
  }
}
}  // namespace

// Returns the max deviation of the emulated readout from the direct simulation, or a negative
// code if the schedule is inconsistent (-1 build failure, -2 address collision).
extern "C" double qp_sched_selftest(int n, int L, int ansatz, unsigned seed) {
  QPSched S;
  if (qp_build_sched(n, L, ansatz, &S) != 0) return -1.0;
  const int lb = S.lb, AMPS = 1 << lb, GL = 1 << (n - lb), PPW = 32 / GL, DIM = 1 << n;
  std::mt19937 rng(seed);
  std::uniform_real_distribution<double> U(-3.0, 3.0);
  std::vector<U2> gates(L * n);
  for (auto& g : gates) {  // RZ(c) RY(b) RZ(a)
    double a = U(rng), b = U(rng), c = U(rng);
    cd ea = std::polar(1.0, -0.5 * (a + c)), eb = std::polar(1.0, 0.5 * (a - c));
    double co = std::cos(0.5 * b), si = std::sin(0.5 * b);
    g = {ea * co, -std::conj(eb) * si, eb * si, std::conj(ea) * co};
  }
  // diagonal phase of each layer (stands in for the CRZ mesh: any diagonal exercises the
  // logical-index tables)
  std::vector<double> dph((size_t)L * DIM);
  for (auto& x : dph) x = U(rng);
  const bool diag = qp_has_crz(ansatz);
  std::vector<std::vector<double>> theta(PPW, std::vector<double>(n));
  for (auto& t : theta)
    for (auto& x : t) x = U(rng);
  std::vector<cd> smem((size_t)PPW * DIM);
  double err = 0.0;
  std::vector<std::vector<double>> zsum(PPW, std::vector<double>(n, 0.0));
  for (int l = 0; l < L; ++l) {
    for (int p = 0; p < S.npl; ++p) {
      const int P = l * S.npl + p;
      std::vector<int> seen((size_t)PPW * DIM, 0);
      for (int lane = 0; lane < 32; ++lane) {
        const int slot = lane / GL;
        cd* st = &smem[(size_t)slot * DIM];
        std::vector<cd> r(AMPS);
        std::vector<int> ad(AMPS);
        for (int j = 0; j < AMPS; ++j) {
          ad[j] = S.lane_addr[P][lane] ^ S.joff[P][j];
          if (ad[j] < 0 || ad[j] >= DIM) return -2.0;
          if (seen[(size_t)slot * DIM + ad[j]]++) return -2.0;
        }
        if (P == 0) {
          uint32_t localmask = 0;
          for (int b = 0; b < lb; ++b) localmask |= 1u << S.ql[0][b];
          cd A = 1.0;
          for (int q = 0; q < n; ++q) {
            if ((localmask >> q) & 1u) continue;
            const int bit = (S.enc_k[lane] >> (n - 1 - q)) & 1;
            const double c = std::cos(0.5 * theta[slot][q]), s = std::sin(0.5 * theta[slot][q]);
            A *= bit ? cd(0, -s) : cd(c, 0);
          }
          for (int j = 0; j < AMPS; ++j) {
            cd B = 1.0;
            for (int b = 0; b < lb; ++b) {
              const int q = S.ql[0][b];
              const double c = std::cos(0.5 * theta[slot][q]), s = std::sin(0.5 * theta[slot][q]);
              B *= ((j >> b) & 1) ? cd(0, -s) : cd(c, 0);
            }
            r[j] = A * B;
          }
        } else {
          for (int j = 0; j < AMPS; ++j) r[j] = st[ad[j]];
        }
        for (int b = 0; b < S.ngate[P]; ++b) {
          const U2& u = gates[l * n + S.ql[P][b]];
          for (int j0 = 0; j0 < AMPS; ++j0) {
            if (j0 & (1 << b)) continue;
            const int j1 = j0 | (1 << b);
            cd x = r[j0], y = r[j1];
            r[j0] = u.a * x + u.b * y;
            r[j1] = u.c * x + u.d * y;
          }
        }
        if (diag && p == S.npl - 1) {
          for (int j = 0; j < AMPS; ++j) {
            const int k = S.klog[l][lane] ^ S.jlog[l][j];
            if (k < 0 || k >= DIM) return -2.0;
            r[j] *= std::polar(1.0, dph[(size_t)l * DIM + k]);
          }
        }
        if (P == L * S.npl - 1) {
          std::vector<double> w(AMPS);
          for (int j = 0; j < AMPS; ++j) w[j] = std::norm(r[j]);
          for (int h = 1; h < AMPS; h <<= 1)
            for (int j = 0; j < AMPS; ++j)
              if (!(j & h)) { double x = w[j], y = w[j | h]; w[j] = x + y; w[j | h] = x - y; }
          for (int i = 0; i < n; ++i) {
            const double sg = ((S.ro_mask[lane] >> i) & 1u) ? -1.0 : 1.0;
            zsum[slot][i] += sg * w[S.ro_sel[i]];
          }
        }
        for (int j = 0; j < AMPS; ++j) st[ad[j]] = r[j];
      }
    }
  }
  for (int slot = 0; slot < PPW; ++slot) {
    std::vector<cd> s(DIM, 0.0);
    s[0] = 1.0;
    for (int q = 0; q < n; ++q) {
      const double c = std::cos(0.5 * theta[slot][q]), si = std::sin(0.5 * theta[slot][q]);
      apply_direct(s, n, q, U2{c, cd(0, -si), cd(0, -si), c});
    }
    for (int l = 0; l < L; ++l) {
      for (int q = 0; q < n; ++q) apply_direct(s, n, q, gates[l * n + q]);
      if (diag) {
        for (int k = 0; k < DIM; ++k) s[k] *= std::polar(1.0, dph[(size_t)l * DIM + k]);
      } else if (ansatz == 6 && n > 1) {
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const int bc = 1 << (n - 1 - i), bt = 1 << (n - 1 - j);
            for (int k = 0; k < DIM; ++k)
              if ((k & bc) && !(k & bt)) std::swap(s[k], s[k | bt]);
          }
      } else if (ansatz != 3 && n > 1) {
        const int r = ansatz == 2 ? 1 + (l % (n - 1)) : 1;
        for (int i = 0; i < n; ++i) {
          const int bc = 1 << (n - 1 - i), bt = 1 << (n - 1 - (i + r) % n);
          for (int k = 0; k < DIM; ++k)
            if ((k & bc) && !(k & bt)) std::swap(s[k], s[k | bt]);
        }
      }
    }
    for (int i = 0; i < n; ++i) {
      double z = 0;
      for (int k = 0; k < DIM; ++k) z += std::norm(s[k]) * (((k >> (n - 1 - i)) & 1) ? -1.0 : 1.0);
      err = std::fmax(err, std::fabs(z - zsum[slot][i]));
    }
  }
  return err;
}

// Planner's worst predicted shared-memory bank-conflict factor for a configuration.
extern "C" int qp_sched_conflicts(int n, int L, int ansatz) {
  QPSched S;
  if (qp_build_sched(n, L, ansatz, &S) != 0) return -1;
  return S.conflict_max;
}
