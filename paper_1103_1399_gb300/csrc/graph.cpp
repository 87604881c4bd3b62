// Device-driven evolution: one CUDA graph runs a whole step range [k0, k1) of
// the streaming pass plan with no host involvement between passes.
//
// Graph (every piece a captured chain of kernel launches):
//   prologue   P row at position 0, low pass W.P (first), the other groups up;
//              the loop counter is zeroed
//   WHILE loop body = kGraphUnroll Strang steps: their B rows and merged P rows
//              (offset by the counter), then per step the phase-group W.B.W
//              pass, the other groups down, the merged low pass, the other
//              groups up; the last node advances the counter and sets the loop
//              condition.  Runs L = (k1 - k0 - 1) / kGraphUnroll times.
//   remainder  the other (k1 - k0 - 1) mod kGraphUnroll merged steps, unrolled
//   epilogue   the last step, ending with the low pass W then P (last)
// The pass order and the phase rows are those of the per-pass launch path
// (build_passes, launch_tables' entry functions), so both give the same state
// bit for bit.  The loop ends because its counter only grows and the condition
// is counter < L * kGraphUnroll.
#include <vector>

#include "engine_internal.h"

namespace qaa {

namespace {

struct Capture {
  cudaStream_t st = nullptr;
  cudaGraph_t g = nullptr;
  ~Capture() {
    if (g) cudaGraphDestroy(g);
    if (st) cudaStreamDestroy(st);
  }
};

// Record launches into `into` (a fresh graph, or a conditional node's body).
template <class F>
cudaError_t capture_into(cudaStream_t st, cudaGraph_t into, F&& body) {
  cudaError_t e = cudaStreamBeginCaptureToGraph(st, into, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  const cudaError_t eb = body();
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(st, &out);
  return eb != cudaSuccess ? eb : e;
}

cudaError_t launch_all(const LaunchCtx& lc, const GraphSpec& s, const std::vector<Pass>& passes) {
  for (const Pass& p : passes) {
    const cudaError_t e =
        launch_planned_pass(lc, *s.plan, p, s.psi, s.m, s.cl, s.prow, s.brow, s.err, s.counts, s.fold);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The low passes of a captured piece end the range's steps first_rel,
// first_rel + 1, ... (their norm-fold slots; build_passes numbers them from
// the piece's own start).  A loop body's pieces start at multiples of
// kGraphUnroll (even), so the slot parity is the same in every iteration.
void number_low_passes(std::vector<Pass>& passes, long long first_rel) {
  long long r = first_rel;
  for (Pass& p : passes)
    if (p.rel >= 0) p.rel = static_cast<int>(r++);
}

}  // namespace

size_t graph_scratch_bytes(int n, int m) {
  const size_t p = static_cast<size_t>(kGraphUnroll + 1) * static_cast<size_t>(m + 1);
  const size_t b = static_cast<size_t>(kGraphUnroll) * static_cast<size_t>(n + 1);
  return 16 + 8 * (p + b);
}

void graph_scratch_split(void* base, int m, GraphSpec& s) {
  char* c = static_cast<char*>(base);
  s.ctr = reinterpret_cast<long long*>(c);
  s.prow = reinterpret_cast<float2*>(c + 16);
  s.brow = s.prow + static_cast<size_t>(kGraphUnroll + 1) * static_cast<size_t>(m + 1);
}

cudaError_t build_evolve_graph(const GraphSpec& s, cudaGraphExec_t* out) {
  *out = nullptr;
  const PassPlan& plan = *s.plan;
  if (plan.onchip || s.k1 <= s.k0) return cudaErrorInvalidValue;
  Capture cap;
  cudaError_t e = cudaStreamCreateWithFlags(&cap.st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaGraphCreate(&cap.g, 0);
  if (e != cudaSuccess) return e;
  const LaunchCtx lc{cap.st, s.num_sms};
  const long long merged = s.k1 - s.k0 - 1;  // steps that end in a merged low pass
  const long long L = merged / kGraphUnroll, R = merged % kGraphUnroll;
  std::vector<Pass> passes;
  auto rows = [&](int dst_p0, long long p_first, int nprow, long long k_first, int nbrow, const long long* ctr) {
    return launch_graph_rows(lc, s.prow, dst_p0, p_first, nprow, s.brow, k_first, nbrow, ctr, plan.n, s.m, s.dt,
                             s.s_dev, s.K, s.k0, s.k1, plan.wht_kind == kRotationForm, s.dt_dev);
  };
  std::vector<cudaGraphNode_t> chain;
  auto add_child = [&](cudaGraph_t child) -> cudaError_t {
    cudaGraphNode_t node = nullptr;
    const cudaError_t ec = cudaGraphAddChildGraphNode(&node, cap.g, chain.empty() ? nullptr : &chain.back(),
                                                      chain.empty() ? 0 : 1, child);
    if (ec == cudaSuccess) chain.push_back(node);
    return ec;
  };
  auto captured_child = [&](auto&& body) -> cudaError_t {
    cudaGraph_t child = nullptr;
    cudaError_t ec = cudaGraphCreate(&child, 0);
    if (ec != cudaSuccess) return ec;
    ec = capture_into(cap.st, child, body);
    if (ec == cudaSuccess) ec = add_child(child);
    cudaGraphDestroy(child);
    return ec;
  };

  // prologue
  e = captured_child([&]() -> cudaError_t {
    cudaError_t ec = cudaMemsetAsync(s.ctr, 0, sizeof(long long), cap.st);
    if (ec == cudaSuccess) ec = rows(0, 0, 1, 0, 0, nullptr);
    build_passes(plan, 0, 1, 0, 0, passes);  // zero steps: the first low pass and the groups up
    return ec == cudaSuccess ? launch_all(lc, s, passes) : ec;
  });
  if (e != cudaSuccess) return e;

  // WHILE loop over blocks of kGraphUnroll merged steps
  if (L > 0) {
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, cap.g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, cap.g, &chain.back(), nullptr, 1, &cp);
    if (e != cudaSuccess) return e;
    chain.push_back(node);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = capture_into(cap.st, body, [&]() -> cudaError_t {
      cudaError_t ec = rows(1, 1, kGraphUnroll, s.k0, kGraphUnroll, s.ctr);
      // kGraphUnroll merged steps: B rows 0.., P rows 1.. (build_passes' chunk convention)
      build_passes(plan, -1, 1ll << 40, 0, kGraphUnroll, passes);
      number_low_passes(passes, 0);
      if (ec == cudaSuccess) ec = launch_all(lc, s, passes);
      if (ec == cudaSuccess) ec = launch_graph_advance(lc, s.ctr, kGraphUnroll, L * kGraphUnroll, h);
      return ec;
    });
    if (e != cudaSuccess) return e;
  }

  // remainder, unrolled
  if (R > 0) {
    e = captured_child([&]() -> cudaError_t {
      const long long off = L * kGraphUnroll;
      cudaError_t ec = rows(1, 1 + off, static_cast<int>(R), s.k0 + off, static_cast<int>(R), nullptr);
      build_passes(plan, -1, 1ll << 40, 0, R, passes);
      number_low_passes(passes, off);
      return ec == cudaSuccess ? launch_all(lc, s, passes) : ec;
    });
    if (e != cudaSuccess) return e;
  }

  // epilogue: the last step (B row of step k1 - 1, P row at position k1 - k0)
  e = captured_child([&]() -> cudaError_t {
    cudaError_t ec = rows(1, s.k1 - s.k0, 1, s.k1 - 1, 1, nullptr);
    build_passes(plan, -1, 1, 0, 1, passes);  // one step, no first pass, ending in the last low pass
    number_low_passes(passes, s.k1 - s.k0 - 1);
    return ec == cudaSuccess ? launch_all(lc, s, passes) : ec;
  });
  if (e != cudaSuccess) return e;

  return cudaGraphInstantiate(out, cap.g, 0);
}

}  // namespace qaa
