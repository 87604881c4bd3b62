// Host check of the norm-fold slot schedule (fold_for in qaa_internal.cuh):
// for every period F and run length K, with the step numbering of per-pass
// launches (step j = j) and of launch graphs (the 8-step loop body numbered
// 0..7 in every iteration, then the remainder and the last step numbered on),
// every low pass that corrects reads the reference written by the range's
// first pass and a measurement slot last written by an earlier pass, at most
// F steps back (the first pass's own copy at step 0, so that step 0's
// correction is exactly 1), and no pass reads a slot it also writes.
// Prints "ok" and exits 0, else prints the first violation and exits 1.
#include <cstdio>
#include <vector>

#include "qaa_internal.cuh"

namespace {

int run(int F, int K, bool graph) {
  static double slots[qaa::kFoldBytes / sizeof(double)];
  float2* base = reinterpret_cast<float2*>(slots);
  auto slot_id = [&](const float2* p) { return p ? static_cast<int>((p - base) / qaa::kFoldSlot) : -1; };
  // last writer (logical step, -1 = the first pass) of each slot; -2 = never
  int writer[3] = {-2, -2, -2};
  const int L = graph ? (K - 1) / 8 : 0;  // loop-body iterations of the graph
  for (int j = -1; j < K; ++j) {
    qaa::Pass p{};
    p.rel = (j >= 0 && j < 8 * L) ? j % 8 : j;
    const qaa::NormFold f = qaa::fold_for(slots, p, F);
    const int out = slot_id(f.out), out2 = slot_id(f.out2), ref = slot_id(f.ref), prev = slot_id(f.prev);
    if ((ref >= 0) != (prev >= 0)) {
      std::printf("F=%d K=%d graph=%d step %d: reference and measurement not read together\n", F, K, graph, j);
      return 1;
    }
    if (j == -1 && (out != 0 || out2 < 0 || ref >= 0)) {
      std::printf("F=%d K=%d graph=%d: the first pass must write the reference and one more slot only\n", F, K,
                  graph);
      return 1;
    }
    if (ref >= 0) {
      if (ref != 0 || writer[0] != -1) {
        std::printf("F=%d K=%d graph=%d step %d: reference not from the first pass\n", F, K, graph, j);
        return 1;
      }
      if (prev == out || prev == out2 || ref == out || ref == out2) {
        std::printf("F=%d K=%d graph=%d step %d: a slot read and written by one pass\n", F, K, graph, j);
        return 1;
      }
      const int w = writer[prev];
      if (w == -2 || w >= j || (j > 0 && w < j - F) || (j == 0 && w != -1)) {
        std::printf("F=%d K=%d graph=%d step %d: measurement slot %d last written by step %d\n", F, K, graph, j,
                    prev, w);
        return 1;
      }
    } else if (j >= 0 && j % F == 0) {
      std::printf("F=%d K=%d graph=%d step %d: no correction where one is due\n", F, K, graph, j);
      return 1;
    }
    if (j >= 0 && (j + 1) % F == 0 && out < 0) {
      std::printf("F=%d K=%d graph=%d step %d: no measurement where one is due\n", F, K, graph, j);
      return 1;
    }
    if (out >= 0) writer[out] = j;
    if (out2 >= 0) writer[out2] = j;
  }
  return 0;
}

}  // namespace

int main() {
  for (int F : {1, 2, 4, 8})
    for (int K = 1; K <= 70; ++K)
      for (bool graph : {false, true})
        if (run(F, K, graph)) return 1;
  // the period by size divides 8 (uniform graph bodies)
  for (int n = 1; n <= 34; ++n)
    if (8 % qaa::fold_period(n) != 0) {
      std::printf("fold_period(%d) = %d does not divide 8\n", n, qaa::fold_period(n));
      return 1;
    }
  std::printf("ok\n");
  return 0;
}
