// sip_shape.cu -- host-side cost model of a sweep launch, used to rank the
// tile shapes of a plan (and the candidates the autotuner times).
//
// A sweep (the forward or backward substitution of Sec. 2, Eqs. 9-10) runs as
// hyperplane wavefronts over 32 x TK column tiles of every block.  The model
// replays one launch: tiles are claimed in the launch's order (anti-diagonal
// waves cj + ck, blocks interleaved) by the resident CTAs, CTA slot s sitting
// on SM s mod nsm; a tile starts once its south neighbour (cj - 1) has walked
// 32 + lead steps and its bottom neighbour (ck - 1) TK + lead steps, and it
// walks nx + njt + nkt - 2 steps.  One step of a tile costs a + b w cycles,
// w the warps per SM sub-partition of all tiles then active on its SM (the
// average over the tile's lifetime, solved by a short fixed-point
// iteration).  a and b were fitted on GB300 to the launches of 256^3, 192^3
// and 128^3 Poisson blocks for every shape with one and two rows per thread.
// Measured against the fastest shape of each launch (128^3, 256^3, the
// 64-block mesh; FP32 and FP64 sweeps) its first choice is the fastest or
// within 7 % (15 % for the FP64 mesh), and the fastest shape is always among
// its first three, which the autotuner then times.
#include <algorithm>
#include <cmath>
#include <queue>
#include <utility>
#include <vector>

#include "sip_internal.h"

namespace sipk {

namespace {

struct StepFit {
  double a, b;  // cycles per step: a + b x (warps per SM sub-partition)
};

StepFit step_fit(int Q, bool fp64) {
  // FP64: one warp's DFMA holds a sub-partition's FP64 pipe for 64 cycles,
  // hence the large per-warp term.  Four rows per thread: measured 1.45x the
  // step of two at equal TK.
  if (fp64) return Q == 1 ? StepFit{620, 340} : Q == 2 ? StepFit{1260, 320} : StepFit{1830, 460};
  return Q == 1 ? StepFit{700, 75} : Q == 2 ? StepFit{910, 70} : StepFit{1320, 100};
}

constexpr double kLead = 4;  // start slack of a tile behind its producers (steps)
constexpr int kIters = 3;

struct MTile {
  int nst;       // steps of the tile's walk
  int upJ, upK;  // claim index of the producers (-1: none)
};

}  // namespace

double sweep_model_cycles(const int *dims, int nblocks, int Q, int NW, int ctas, int nsm, bool fp64) {
  if (nblocks <= 0 || Q <= 0 || NW <= 0 || ctas <= 0 || nsm <= 0) return -1;
  const int TK = Q * NW;
  // claim order of the launch
  std::vector<int> nTJ(nblocks), nTK(nblocks);
  int maxwave = 0;
  for (int b = 0; b < nblocks; ++b) {
    const int ny = dims[3 * b + 1], nz = dims[3 * b + 2];
    if (dims[3 * b] <= 0 || ny <= 0 || nz <= 0) return -1;
    nTJ[b] = (ny + kTJ - 1) / kTJ;
    nTK[b] = (nz + TK - 1) / TK;
    maxwave = std::max(maxwave, nTJ[b] + nTK[b] - 2);
  }
  std::vector<std::vector<int>> pos(nblocks);
  for (int b = 0; b < nblocks; ++b) pos[b].assign((size_t)nTJ[b] * nTK[b], -1);
  std::vector<MTile> t;
  for (int w = 0; w <= maxwave; ++w)
    for (int b = 0; b < nblocks; ++b)
      for (int ck = 0; ck < nTK[b]; ++ck) {
        const int cj = w - ck;
        if (cj < 0 || cj >= nTJ[b]) continue;
        const int nx = dims[3 * b], ny = dims[3 * b + 1], nz = dims[3 * b + 2];
        const int njt = std::min(kTJ, ny - kTJ * cj), nkt = std::min(TK, nz - TK * ck);
        MTile m;
        m.nst = nx + njt + nkt - 2;
        m.upJ = cj > 0 ? pos[b][(size_t)ck * nTJ[b] + cj - 1] : -1;
        m.upK = ck > 0 ? pos[b][(size_t)(ck - 1) * nTJ[b] + cj] : -1;
        pos[b][(size_t)ck * nTJ[b] + cj] = (int)t.size();
        t.push_back(m);
      }
  const int n = (int)t.size();
  const int grid = std::min(n, ctas);
  const StepFit fit = step_fit(Q, fp64);
  const double wq = std::ceil(NW / 4.0);  // warps per sub-partition of one tile
  std::vector<double> L(n, fit.a + fit.b * wq), S(n), F(n);
  std::vector<int> sm(n);
  double makespan = 0;
  for (int it = 0; it < kIters; ++it) {
    // replay the claims: a free CTA slot takes the next tile
    using Slot = std::pair<double, int>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> freeq;
    for (int s = 0; s < grid; ++s) freeq.push({0.0, s});
    makespan = 0;
    for (int m = 0; m < n; ++m) {
      const Slot sl = freeq.top();
      freeq.pop();
      double st = sl.first, fin = 0;
      if (t[m].upJ >= 0) {
        const int u = t[m].upJ;
        st = std::max(st, S[u] + (kTJ + kLead) * L[u]);
        fin = std::max(fin, F[u] + kLead * L[m]);
      }
      if (t[m].upK >= 0) {
        const int u = t[m].upK;
        st = std::max(st, S[u] + (TK + kLead) * L[u]);
        fin = std::max(fin, F[u] + kLead * L[m]);
      }
      S[m] = st;
      F[m] = std::max(st + t[m].nst * L[m], fin);
      sm[m] = sl.second % nsm;
      freeq.push({F[m], sl.second});
      makespan = std::max(makespan, F[m]);
    }
    if (it + 1 == kIters) break;
    // tiles active on each SM over time: integral of the active count over
    // each tile's lifetime (sweep over sorted start / end events)
    std::vector<std::vector<int>> bysm(nsm);
    for (int m = 0; m < n; ++m) bysm[sm[m]].push_back(m);
    for (auto &ms : bysm) {
      if (ms.empty()) continue;
      std::vector<std::pair<double, int>> ev;
      ev.reserve(2 * ms.size());
      for (int m : ms) {
        ev.push_back({S[m], +1});
        ev.push_back({F[m], -1});
      }
      std::sort(ev.begin(), ev.end());
      // tx[q]: time of event q; acc[q]: integral of the active count up to
      // tx[q]; after[q]: the count right after event q
      std::vector<double> tx(ev.size()), acc(ev.size());
      std::vector<int> after(ev.size());
      int active = 0;
      double a = 0;
      for (size_t q = 0; q < ev.size(); ++q) {
        if (q > 0) a += active * (ev[q].first - ev[q - 1].first);
        tx[q] = ev[q].first;
        acc[q] = a;
        active += ev[q].second;
        after[q] = active;
      }
      auto at = [&](double x) {  // integral of the active count up to x
        const size_t q = std::upper_bound(tx.begin(), tx.end(), x) - tx.begin();
        return q == 0 ? 0.0 : acc[q - 1] + after[q - 1] * (x - tx[q - 1]);
      };
      for (int m : ms) {
        const double dur = F[m] - S[m];
        if (dur <= 0) continue;
        const double conc = std::max(1.0, (at(F[m]) - at(S[m])) / dur);
        L[m] = 0.5 * L[m] + 0.5 * (fit.a + fit.b * wq * conc);
      }
    }
  }
  return makespan;
}

}  // namespace sipk
