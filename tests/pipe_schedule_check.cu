// Host-side check of the pipelined middle passes' dispenser order
// (make_pipe_sched / pipe_decode in passes7.cuh): over many schedule shapes,
// every (kind, plane, tile) item appears exactly once, within range, every
// plane's row-forward items come before its middle items and those before
// its row-inverse items (the order a CTA's waits rely on).  Prints
// "cases N bad B" and exits non-zero on any violation.
#include <cstdio>
#include <vector>

#include "../paper_2504_19410_gb300/csrc/passes7.cuh"

using namespace fsa;

int main() {
  int bad = 0, cases = 0;
  for (int a : {1, 8, 12, 16, 32})
    for (int b : {16, 24, 32})
      for (int NP : {2, 3, 5, 65, 257, 514, 16448})
        for (int L : {1, 2, 3, 8, 17, 40}) {
          if (2 * L > NP) continue;
          const int c = a;
          const PipeSched s = make_pipe_sched(a, b, c, NP, L);
          ++cases;
          if (s.total != NP * (a + b + c)) {
            ++bad;
            continue;
          }
          std::vector<long long> rf_last(NP, -1), mid_first(NP, 1LL << 60), mid_last(NP, -1), ri_first(NP, 1LL << 60);
          std::vector<int> seen((size_t)NP * (a + b + c), 0);
          for (int i = 0; i < s.total; ++i) {
            int kind, plane, tile;
            pipe_decode(s, i, kind, plane, tile);
            const int lim = kind == 0 ? a : kind == 1 ? b : c;
            if (kind < 0 || kind > 2 || plane < 0 || plane >= NP || tile < 0 || tile >= lim) {
              ++bad;
              break;
            }
            seen[(size_t)plane * (a + b + c) + (kind == 0 ? 0 : kind == 1 ? a : a + b) + tile]++;
            if (kind == 0 && i > rf_last[plane]) rf_last[plane] = i;
            if (kind == 1 && i < mid_first[plane]) mid_first[plane] = i;
            if (kind == 1 && i > mid_last[plane]) mid_last[plane] = i;
            if (kind == 2 && i < ri_first[plane]) ri_first[plane] = i;
          }
          for (int v : seen)
            if (v != 1) {
              ++bad;
              break;
            }
          for (int q = 0; q < NP; ++q)
            if (!(rf_last[q] < mid_first[q]) || !(mid_last[q] < ri_first[q])) {
              ++bad;
              break;
            }
        }
  std::printf("cases %d bad %d\n", cases, bad);
  return bad != 0;
}
