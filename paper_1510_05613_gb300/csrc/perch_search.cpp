// Tree search over the Monotone Scene Generation Tree (Sec. IV-A/B), driven
// by batched successor evaluation on the device.
//
// Uniform-cost search (Alg. 1 with the admissible anchor heuristic h0 = 0
// and w = 1): states are keyed by the sorted multiset of their objects (the
// same set in another order has the same render and the same cost-to-go, so
// the paper keeps one ordering), the cheapest g per key is kept, and a state
// reached later with a smaller g is reopened. Up to `batch_states` open states
// are expanded per device launch: every state popped has g <= the best goal
// found so far, and the search ends only when the smallest open g exceeds it,
// so batching never changes the answer (edge costs are non-negative). Among
// goals of minimum cost the lexicographically smallest sorted key is returned.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <functional>
#include <limits>
#include <queue>
#include <unordered_map>
#include <vector>

#include "perch_ctx.h"

namespace {

using Key = std::vector<uint64_t>;

uint64_t pack(const perch_obj& o) {
  return ((uint64_t)o.mesh << 48) | ((uint64_t)(uint16_t)o.ix << 32) | ((uint64_t)(uint16_t)o.iy << 16) |
         (uint64_t)o.iyaw;
}

perch_obj unpack(uint64_t k) {
  perch_obj o;
  o.mesh = (uint16_t)(k >> 48);
  o.ix = (int16_t)(uint16_t)(k >> 32);
  o.iy = (int16_t)(uint16_t)(k >> 16);
  o.iyaw = (uint16_t)k;
  return o;
}

struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = 1469598103934665603ULL;
    for (uint64_t x : k) {
      h ^= x + 0x9E3779B97F4A7C15ULL + (h << 6) + (h >> 2);
      h *= 1099511628211ULL;
    }
    return (size_t)h;
  }
};

struct State {
  Key key;
  int64_t g;
  bool closed;
};

struct OpenEntry {
  int64_t g;
  int idx;
};

}  // namespace

extern "C" int perch_search(perch_ctx* ctx, const perch_search_params* prm, perch_result* res) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!prm || !res || prm->K < 1 || prm->K > 16 || !prm->mesh_multiset || prm->batch_states < 1)
    return ctx->fail(PERCH_E_ARG, "search: bad parameters");
  if (!(prm->w >= 1.0f)) return ctx->fail(PERCH_E_ARG, "search: w must be >= 1");
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  const int K = prm->K;
  for (int i = 0; i < K; ++i)
    if (prm->mesh_multiset[i] >= ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "search: mesh %d out of range", i);
  std::memset(res, 0, sizeof *res);
  res->cost = -1;
  const auto t0 = std::chrono::steady_clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };

  std::vector<State> states;
  std::unordered_map<Key, int, KeyHash> index;
  std::vector<OpenEntry> heap;
  // min-heap on (g, key)
  auto worse = [&](const OpenEntry& a, const OpenEntry& b) {
    if (a.g != b.g) return a.g > b.g;
    return states[a.idx].key > states[b.idx].key;
  };
  states.push_back(State{Key{}, 0, false});
  index[Key{}] = 0;
  heap.push_back(OpenEntry{0, 0});

  const int64_t INF = std::numeric_limits<int64_t>::max();
  int64_t best_g = INF;
  Key best_key;
  int64_t expansions = 0, successors = 0;
  const int n_poses_per_type = ctx->nx * ctx->ny * ctx->n_yaw;
  const int B = std::min(prm->batch_states, std::max(1, 65535 / std::max(K - 1, 1)));
  int status = PERCH_OK;

  std::vector<perch_obj> parents, hyps;
  std::vector<int32_t> plen, hparent;
  std::vector<perch_cost> out;
  std::vector<int> batch;
  while (!heap.empty()) {
    if ((prm->time_limit_s > 0 && elapsed() > prm->time_limit_s) ||
        (prm->max_expansions > 0 && expansions >= prm->max_expansions)) {
      status = PERCH_E_TIMEOUT;
      break;
    }
    batch.clear();
    while (!heap.empty() && (int)batch.size() < B) {
      const OpenEntry top = heap.front();
      if (top.g > best_g) break;
      std::pop_heap(heap.begin(), heap.end(), worse);
      heap.pop_back();
      State& s = states[top.idx];
      if (s.closed || top.g > s.g) continue;  // stale entry
      s.closed = true;
      batch.push_back(top.idx);
    }
    if (batch.empty()) {
      if (heap.empty() || heap.front().g > best_g) break;
      continue;
    }
    // successors of the batch: distinct unplaced types x every pose (Eq. (3))
    const int stride = std::max(K - 1, 1);
    parents.assign((size_t)batch.size() * stride, perch_obj{0, 0, 0, 0});
    plen.assign(batch.size(), 0);
    hyps.clear();
    hparent.clear();
    for (size_t bi = 0; bi < batch.size(); ++bi) {
      const Key& key = states[batch[bi]].key;
      plen[bi] = (int32_t)key.size();
      std::vector<int> remaining(prm->mesh_multiset, prm->mesh_multiset + K);
      for (size_t j = 0; j < key.size(); ++j) {
        parents[bi * stride + j] = unpack(key[j]);
        auto it = std::find(remaining.begin(), remaining.end(), (int)(key[j] >> 48));
        if (it != remaining.end()) remaining.erase(it);
      }
      std::sort(remaining.begin(), remaining.end());
      remaining.erase(std::unique(remaining.begin(), remaining.end()), remaining.end());
      for (int m : remaining)
        for (int ix = 0; ix < ctx->nx; ++ix)
          for (int iy = 0; iy < ctx->ny; ++iy)
            for (int k = 0; k < ctx->n_yaw; ++k) {
              hyps.push_back(perch_obj{(uint16_t)m, (uint16_t)k, (int16_t)ix, (int16_t)iy});
              hparent.push_back((int32_t)bi);
            }
    }
    (void)n_poses_per_type;
    out.resize(hyps.size());
    int rc = perch_eval_successors(ctx, parents.data(), stride, plen.data(), (int32_t)batch.size(), hparent.data(),
                                   hyps.data(), (int64_t)hyps.size(), K, out.data());
    if (rc != PERCH_OK) return rc;
    expansions += (int64_t)batch.size();
    successors += (int64_t)hyps.size();
    for (size_t h = 0; h < hyps.size(); ++h) {
      const perch_cost& r = out[h];
      if (r.viol > 0) continue;  // occludes the parent: not a successor
      const int pidx = batch[hparent[h]];
      const int64_t ng = states[pidx].g + (int64_t)r.djr + r.djo + r.resid;
      if (ng > best_g) continue;
      Key ck = states[pidx].key;
      ck.insert(std::upper_bound(ck.begin(), ck.end(), pack(hyps[h])), pack(hyps[h]));
      if ((int)ck.size() == K) {
        if (ng < best_g || (ng == best_g && ck < best_key)) {
          best_g = ng;
          best_key = ck;
        }
        continue;
      }
      auto it = index.find(ck);
      if (it == index.end()) {
        const int idx = (int)states.size();
        states.push_back(State{std::move(ck), ng, false});
        index.emplace(states[idx].key, idx);
        heap.push_back(OpenEntry{ng, idx});
        std::push_heap(heap.begin(), heap.end(), worse);
      } else {
        State& s = states[it->second];
        if (ng < s.g) {
          s.g = ng;
          s.closed = false;  // a cheaper way in: reopen
          heap.push_back(OpenEntry{ng, it->second});
          std::push_heap(heap.begin(), heap.end(), worse);
        }
      }
    }
  }
  res->expansions = expansions;
  res->successors = successors;
  res->seconds = elapsed();
  if (best_g != INF) {
    res->cost = best_g;
    res->n_objs = (int32_t)best_key.size();
    for (size_t j = 0; j < best_key.size(); ++j) res->objs[j] = unpack(best_key[j]);
  }
  res->proven_optimal = (status == PERCH_OK && best_g != INF) ? 1 : 0;
  if (status == PERCH_E_TIMEOUT) return ctx->fail(PERCH_E_TIMEOUT, "search limit reached; best so far returned");
  if (best_g == INF) return ctx->fail(PERCH_E_RANGE, "no valid complete scene exists in the tree");
  return PERCH_OK;
}
