// Batched-processing schedule of a processing graph (Sec. 4, Alg. 1 lines 1-4), host code.
//
// A schedule is a sequence of types t_0 .. t_N; step n computes the maximal subset V_n of the not yet
// computed nodes of type t_n whose predecessors are all computed, so the subsets partition the graph, are
// causal and homogeneous.  ScheduleBatchedProcessing: greedy (the type with the most computable nodes,
// ties to the smaller type code) or a layered beam search that keeps the beam_width states with the most
// computed nodes per depth and stops at the first depth that completes the graph (exact shortest schedule
// when the beam holds every state of a depth).  OptimizeNodeOrder: nodes sorted by (step, index), so every
// subset, its parameters and its outputs are one contiguous slice.  GetReadWriteIndex: per step the gather
// list (predecessor position -> consumer position) in the new order, and the store slice.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <unordered_set>
#include <vector>

#include "../../include/mixgraph.h"

namespace {

struct Graph {
  int n = 0;
  std::vector<int> type;
  std::vector<std::vector<int>> succ;
  std::vector<int> indeg;
  std::vector<int> types;   // distinct type codes, ascending
};

struct State {
  std::vector<uint8_t> done;
  std::vector<int> missing;   // predecessors not yet computed
  std::vector<int> seq;
  int ndone = 0;
};

// nodes of type t computable in s
void ready(const Graph& g, const State& s, int t, std::vector<int>& out) {
  out.clear();
  for (int v = 0; v < g.n; ++v)
    if (!s.done[v] && g.type[v] == t && s.missing[v] == 0) out.push_back(v);
}

void apply(const Graph& g, State& s, int t, const std::vector<int>& sub) {
  for (int v : sub) {
    s.done[v] = 1;
    for (int w : g.succ[v]) --s.missing[w];
  }
  s.ndone += (int)sub.size();
  s.seq.push_back(t);
}

uint64_t state_hash(const State& s) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < s.done.size(); ++i)
    if (s.done[i]) h = (h ^ (uint64_t)i) * 1099511628211ull;
  return h;
}

}  // namespace

extern "C" {

mg_status mg_schedule_graph(const int32_t* node_type, int32_t n_nodes, const int32_t* edge_src,
                            const int32_t* edge_dst, int32_t n_edges, int32_t method, int32_t beam_width,
                            int32_t* step_type, int32_t* n_steps, int32_t* node_step, int32_t* order) {
  if (n_nodes < 0 || n_edges < 0 || (n_nodes && !node_type) || (n_edges && (!edge_src || !edge_dst)) ||
      !n_steps || (n_nodes && (!step_type || !node_step || !order)))
    return MG_ERR_INVALID;
  if (method != MG_SCHED_GREEDY && method != MG_SCHED_BEAM) return MG_ERR_INVALID;
  if (method == MG_SCHED_BEAM && beam_width < 1) return MG_ERR_INVALID;
  Graph g;
  g.n = n_nodes;
  g.type.assign(node_type, node_type + n_nodes);
  g.succ.assign(n_nodes, {});
  g.indeg.assign(n_nodes, 0);
  for (int e = 0; e < n_edges; ++e) {
    const int u = edge_src[e], v = edge_dst[e];
    if (u < 0 || u >= n_nodes || v < 0 || v >= n_nodes || u == v) return MG_ERR_INVALID;
    g.succ[u].push_back(v);
    ++g.indeg[v];
  }
  g.types = g.type;
  std::sort(g.types.begin(), g.types.end());
  g.types.erase(std::unique(g.types.begin(), g.types.end()), g.types.end());
  State s0;
  s0.done.assign(n_nodes, 0);
  s0.missing = g.indeg;

  std::vector<int> sub;
  State best;
  bool found = n_nodes == 0;
  if (found) best = s0;
  if (method == MG_SCHED_GREEDY) {
    State s = s0;
    while (s.ndone < n_nodes) {
      int bt = -1;
      size_t bc = 0;
      for (int t : g.types) {
        ready(g, s, t, sub);
        if (sub.size() > bc) {
          bc = sub.size();
          bt = t;
        }
      }
      if (bt < 0) return MG_ERR_INVALID;   // a cycle: nothing computable
      ready(g, s, bt, sub);
      apply(g, s, bt, sub);
    }
    best = s;
    found = true;
  } else {
    std::vector<State> layer{s0};
    while (!found) {
      std::vector<State> next;
      std::unordered_set<uint64_t> seen;
      for (const State& s : layer)
        for (int t : g.types) {
          ready(g, s, t, sub);
          if (sub.empty()) continue;
          State c = s;
          apply(g, c, t, sub);
          if (!seen.insert(state_hash(c)).second) continue;
          next.push_back(std::move(c));
        }
      if (next.empty()) return MG_ERR_INVALID;   // a cycle
      // most computed nodes first; ties by the type sequence (deterministic)
      std::stable_sort(next.begin(), next.end(), [](const State& a, const State& b) {
        if (a.ndone != b.ndone) return a.ndone > b.ndone;
        return a.seq < b.seq;
      });
      if (next.front().ndone == n_nodes) {
        best = next.front();
        found = true;
        break;
      }
      if ((int)next.size() > beam_width) next.resize(beam_width);
      layer.swap(next);
    }
  }
  // replay the sequence for the node steps, then the order
  State s = s0;
  for (size_t k = 0; k < best.seq.size(); ++k) {
    ready(g, s, best.seq[k], sub);
    for (int v : sub) node_step[v] = (int32_t)k;
    apply(g, s, best.seq[k], sub);
    step_type[k] = best.seq[k];
  }
  *n_steps = (int32_t)best.seq.size();
  std::vector<int> idx(n_nodes);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return node_step[a] < node_step[b]; });
  for (int i = 0; i < n_nodes; ++i) order[i] = idx[i];
  return MG_OK;
}

mg_status mg_schedule_io(const int32_t* node_step, const int32_t* order, int32_t n_nodes, int32_t n_steps,
                         const int32_t* edge_src, const int32_t* edge_dst, int32_t n_edges, int32_t* step_begin,
                         int32_t* gather_begin, int32_t* gather_src, int32_t* gather_dst) {
  if (n_nodes < 0 || n_steps < 0 || n_edges < 0 || !step_begin || !gather_begin ||
      (n_nodes && (!node_step || !order)) || (n_edges && (!edge_src || !edge_dst || !gather_src || !gather_dst)))
    return MG_ERR_INVALID;
  std::vector<int> pos(n_nodes, -1);
  for (int i = 0; i < n_nodes; ++i) {
    if (order[i] < 0 || order[i] >= n_nodes || pos[order[i]] >= 0) return MG_ERR_INVALID;
    pos[order[i]] = i;
  }
  std::fill(step_begin, step_begin + n_steps + 1, 0);
  for (int v = 0; v < n_nodes; ++v) {
    if (node_step[v] < 0 || node_step[v] >= n_steps) return MG_ERR_INVALID;
    ++step_begin[node_step[v] + 1];
  }
  for (int k = 0; k < n_steps; ++k) step_begin[k + 1] += step_begin[k];
  // gather lists grouped by the consumer's step, then consumer position, then producer position
  std::vector<int> e(n_edges);
  std::iota(e.begin(), e.end(), 0);
  for (int i = 0; i < n_edges; ++i)
    if (edge_src[i] < 0 || edge_src[i] >= n_nodes || edge_dst[i] < 0 || edge_dst[i] >= n_nodes) return MG_ERR_INVALID;
  std::sort(e.begin(), e.end(), [&](int a, int b) {
    const int sa = node_step[edge_dst[a]], sb = node_step[edge_dst[b]];
    if (sa != sb) return sa < sb;
    if (pos[edge_dst[a]] != pos[edge_dst[b]]) return pos[edge_dst[a]] < pos[edge_dst[b]];
    return pos[edge_src[a]] < pos[edge_src[b]];
  });
  std::fill(gather_begin, gather_begin + n_steps + 1, 0);
  for (int i = 0; i < n_edges; ++i) {
    gather_src[i] = pos[edge_src[e[i]]];
    gather_dst[i] = pos[edge_dst[e[i]]];
    ++gather_begin[node_step[edge_dst[e[i]]] + 1];
  }
  for (int k = 0; k < n_steps; ++k) gather_begin[k + 1] += gather_begin[k];
  return MG_OK;
}

}  // extern "C"
