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
//
// perch_search_multi runs one such search per scene and packs the expansions
// of all unfinished scenes into shared evaluation launches.
//
// Learned queue (heuristics bit 2 or 3, not in the paper's experiments):
// every expansion keeps, per remaining object type, its `n_candidates`
// cheapest valid placements and their exact edge costs. A child s' gets the
// free estimate h_free(s') = sum over its remaining objects of the cheapest
// exact cost of that type at the parent, and the learned estimate
// h_cnn(s') = sum over the remaining objects of min over the parent's
// candidates of that type of (exp(prediction) - 1), the network's edge-cost
// estimate with s' itself as the parent (its z-buffer in the crop). h_cnn
// takes a forward pass, so states are scored lazily: each round the queue
// takes a pool of its front states (max(16, 2 batch_states)), scores the
// unscored ones in one batch across scenes, expands the pool's best
// batch_states states and returns the rest.
//   bit 2: the queue is ordered by g + h_free across depths (ties: deeper
//          first) and the pool's states are expanded in order of g + h_cnn,
//          both estimates of the cost of the whole scene, so the network's
//          ranking decides between states of any depth.
//   bit 3: the queue is ordered deepest first, then by g + h_free, and the
//          pool is re-ranked by g + h_cnn only within a depth (a depth-first
//          dive that the network steers among siblings).
//
// Incumbent (heuristics bit 4, with any of the above or none): before the
// search proper, a greedy completion from the root expands, at each depth,
// the cheapest valid child of the state it expanded last (ties: the smallest
// key), K expansions in all, one per round. Its goal is the first best goal:
// from then on every successor dearer than it is dropped when its record is
// absorbed, instead of entering the open set. Every state the greedy
// completion expands is a state of the tree, expanded at its current g (a
// cheaper way in later reopens it), so the search returns what it returns
// without it; only the open set it has to hold shrinks.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "perch_ctx.h"

namespace {

using Key = std::vector<uint64_t>;
using Clock = std::chrono::steady_clock;
constexpr int64_t kInf = std::numeric_limits<int64_t>::max();
// batches of at least this many hypotheses are built and absorbed by host
// threads (OpenMP), one expanded state or one scene per task
constexpr size_t kParallelMin = 65536;
// record flags that mean "no cost computed": a bounded wait gave up, or an
// index check failed on the device
constexpr uint32_t kNoCost = perch::kFlagTimeout | perch::kFlagBadIndex;

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

// Order-independent hash of an object multiset: the sum (mod 2^64) of a
// SplitMix64 finaliser of each packed object, in two independent variants.
// A state's hash is its parent's plus the added object's, so it costs O(1);
// equal hashes are confirmed by comparing the objects themselves, so the
// hash only speeds up duplicate detection and never decides it.
uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
uint64_t zobj0(uint64_t o) { return mix64(o); }
uint64_t zobj1(uint64_t o) { return mix64(o ^ 0xD1B54A32D192ED03ULL); }

// A state is its predecessor `link` plus one object (the root has none), so
// its key (sorted objects) is rebuilt by walking at most K links.
struct State {
  int64_t g;
  int64_t h_overlap;  // observed points outside the volumes of the state's objects
  int64_t h_free = 0; // learned queue pool key part (see header)
  double h_cnn = -1;  // < 0: not scored yet
  uint64_t hk0 = 0, hk1 = 0;  // multiset hash
  uint64_t obj = 0;   // packed object added to `link`
  int link = -1;      // the state this one extends (fixed at creation)
  int parent = -1;    // state whose expansion generated the cheapest known way in
  int exp = -1;       // this state's own expansion record (learned queue)
  uint8_t depth = 0;  // number of objects
  bool closed = false;
};

// Open-addressing table from a state's first hash to its index (entries with
// equal hashes sit in the same probe run; every match is confirmed).
struct StateIndex {
  std::vector<uint64_t> h;
  std::vector<int32_t> idx;  // -1: empty
  size_t n = 0;
  void init(size_t cap) {
    h.assign(cap, 0);
    idx.assign(cap, -1);
    n = 0;
  }
  template <typename Eq>
  int find(uint64_t key, Eq eq) const {
    const size_t mask = h.size() - 1;
    for (size_t i = key & mask;; i = (i + 1) & mask) {
      if (idx[i] < 0) return -1;
      if (h[i] == key && eq(idx[i])) return idx[i];
    }
  }
  void insert(uint64_t key, int v) {
    if (2 * (n + 1) > h.size()) grow();
    const size_t mask = h.size() - 1;
    size_t i = key & mask;
    while (idx[i] >= 0) i = (i + 1) & mask;
    h[i] = key;
    idx[i] = v;
    ++n;
  }
  void grow() {
    std::vector<uint64_t> oh = std::move(h);
    std::vector<int32_t> oi = std::move(idx);
    init(oh.size() * 2);
    for (size_t i = 0; i < oh.size(); ++i)
      if (oi[i] >= 0) insert(oh[i], oi[i]);
  }
};

// What the learned queue keeps of one expansion: per distinct remaining type,
// up to T cheapest valid placements (mesh = 0xffff pads) and the cheapest cost.
struct ExpansionRecord {
  std::vector<int> types;
  std::vector<perch_obj> top;  // types.size() x T
  std::vector<int64_t> best;   // per type; kInf if no valid placement
  int64_t total = 0;           // sum over the remaining objects (with multiplicity) of best (or a penalty)
};

struct HEntry {  // entry of an inadmissible queue
  int64_t h, g;
  int idx;
};

struct OpenEntry {
  int64_t g;
  int idx;
  int depth;  // ties in g: deeper states first (complete scenes, hence pruning bounds, come early)
};

// One scene's search: uniform-cost search for w = 1 without heuristics,
// Focal-MHA* otherwise (Sec. IV-B, Alg. 1): the anchor queue is keyed by
// g + h0 with h0 = 0; states whose g is within w times the smallest anchor
// key (the focal set) are also ordered by each inadmissible heuristic
// (h_depth = K - |s|, h_overlap = |I| - |I n V_j|, Sec. IV-C), and every round
// expands states from the anchor and from each heuristic queue. The search
// stops once its best goal has g <= w * (smallest anchor key), which is at
// most w * OPT (Theorem 2).
struct SceneSearch {
  int scene = 0, K = 0;
  std::vector<int> multiset;
  std::vector<State> states;
  StateIndex index;
  std::vector<OpenEntry> heap;  // anchor
  int64_t best_g = kInf;
  Key best_key;
  int64_t expansions = 0, successors = 0;
  bool done = false;
  double seconds = 0.0;
  double w = 1.0;
  int heur = 0;                        // bit 0: h_depth, bit 1: h_overlap, bit 2 / 3: learned
  std::vector<OpenEntry> pending;      // generated, not yet in the focal set (min g)
  std::vector<HEntry> hq[3];           // focal states ordered by each heuristic
  std::vector<ExpansionRecord> exps;   // learned queue: one per expanded state
  std::vector<int> pool;               // learned queue: candidates of the current step
  int T = 16;                          // learned queue: placements kept per type
  bool bad_record = false;             // a record carried no cost (flags bit 30 or 31)
  double now = 0.0;                    // seconds since the start, when the current records arrived
  double found_seconds = 0.0;          // when best_key was last set
  int64_t found_expansions = 0;
  // greedy completion (heuristics bit 4): the state it expands next, the
  // state it expands this round, and that state's cheapest child so far
  bool diving = false;
  int dive_next = -1, dive_from = -1, dive_pick = -1;
  int64_t dive_pick_g = kInf;
  bool focal() const { return w > 1.0 || (heur & 15) != 0; }
  bool learned() const { return (heur & 12) != 0; }
  bool dive() const { return (heur & 8) != 0; }  // the depth-first learned queue
  int64_t hval(int which, int idx) const {
    if (which == 2) {
      const int64_t f = std::min<int64_t>(states[idx].g + states[idx].h_free, ((int64_t)1 << 40) - 1);
      if (dive()) return ((int64_t)(K - (int)states[idx].depth) << 40) | f;  // deepest first, then g + h_free
      return (f << 5) | (int64_t)(31 - std::min<int>(states[idx].depth, 31));  // g + h_free; ties: deeper first
    }
    return which == 0 ? (int64_t)(K - (int)states[idx].depth) : states[idx].h_overlap;
  }
  static bool hworse(const HEntry& a, const HEntry& b) {
    if (a.h != b.h) return a.h > b.h;
    if (a.g != b.g) return a.g > b.g;
    return a.idx > b.idx;
  }
  static bool gworse(const OpenEntry& a, const OpenEntry& b) {
    if (a.g != b.g) return a.g > b.g;
    if (a.depth != b.depth) return a.depth < b.depth;
    return a.idx > b.idx;
  }
  void add_open(int64_t g, int idx) {
    push(g, idx);
    if (focal()) {
      pending.push_back(OpenEntry{g, idx, states[idx].depth});
      std::push_heap(pending.begin(), pending.end(), gworse);
    }
  }
  bool stale(const OpenEntry& e) const { return states[e.idx].closed || e.g > states[e.idx].g; }

  bool worse(const OpenEntry& a, const OpenEntry& b) const { return gworse(a, b); }
  // the sorted objects of state idx
  Key key_of(int idx) const {
    Key k;
    for (int i = idx; i > 0; i = states[i].link) k.push_back(states[i].obj);
    std::sort(k.begin(), k.end());
    return k;
  }
  // is state idx the multiset key(pidx) + {o}?
  bool same_set(int idx, int pidx, uint64_t o) const {
    if (states[idx].depth != states[pidx].depth + 1) return false;
    uint64_t a[17], b[17];
    int na = 0, nb = 0;
    for (int i = idx; i > 0; i = states[i].link) a[na++] = states[i].obj;
    for (int i = pidx; i > 0; i = states[i].link) b[nb++] = states[i].obj;
    b[nb++] = o;
    std::sort(a, a + na);
    std::sort(b, b + nb);
    return std::equal(a, a + na, b);
  }
  void push(int64_t g, int idx) {
    heap.push_back(OpenEntry{g, idx, states[idx].depth});
    std::push_heap(heap.begin(), heap.end(), [this](const OpenEntry& a, const OpenEntry& b) { return worse(a, b); });
  }
  void init(int sc, int k, const uint16_t* ms, double w_, int heur_, int64_t n_obs) {
    scene = sc;
    K = k;
    w = w_;
    heur = heur_;
    multiset.assign(ms, ms + k);
    State root;
    root.g = 0;
    root.h_overlap = n_obs;
    states.push_back(root);
    index.init(1 << 16);  // the root is never looked up (no child has depth 0)
    add_open(0, 0);
    diving = (heur & 16) != 0 && K > 1;
    dive_next = diving ? 0 : -1;
  }
  // greedy completion: after a round's records, continue from the cheapest
  // child of the state it expanded, or stop (a goal was reached, or no child
  // was valid)
  void end_round() {
    if (dive_from < 0) return;
    if (dive_pick >= 0 && best_g == kInf && (int)states[dive_pick].depth < K) {
      dive_next = dive_pick;
    } else {
      diving = false;
    }
    dive_from = dive_pick = -1;
    dive_pick_g = kInf;
  }
  // Focal-MHA* round: up to B states from the anchor and from each queue
  void pop_focal(int B, std::vector<int>& out) {
    auto cmp = [this](const OpenEntry& a, const OpenEntry& b) { return worse(a, b); };
    while (!heap.empty() && stale(heap.front())) {
      std::pop_heap(heap.begin(), heap.end(), cmp);
      heap.pop_back();
    }
    if (heap.empty()) {
      done = true;
      return;
    }
    const int64_t f0 = heap.front().g;
    const double bound = w * (double)f0;
    if (best_g != kInf && (double)best_g <= bound) {  // within w * OPT
      done = true;
      return;
    }
    while (!pending.empty() && (double)pending.front().g <= bound) {  // admit into the focal set
      const OpenEntry e = pending.front();
      std::pop_heap(pending.begin(), pending.end(), gworse);
      pending.pop_back();
      if (stale(e)) continue;
      for (int q = 0; q < 3; ++q)
        if (q == 2 ? learned() : (heur & (1 << q)) != 0) {
          hq[q].push_back(HEntry{hval(q, e.idx), e.g, e.idx});
          std::push_heap(hq[q].begin(), hq[q].end(), hworse);
        }
    }
    for (int n = 0; n < B && !heap.empty();) {  // anchor
      const OpenEntry top = heap.front();
      std::pop_heap(heap.begin(), heap.end(), cmp);
      heap.pop_back();
      if (stale(top) || top.g > best_g) continue;
      states[top.idx].closed = true;
      out.push_back(top.idx);
      ++n;
    }
    for (int q = 0; q < 2; ++q) {
      if (!(heur & (1 << q))) continue;
      for (int n = 0; n < B && !hq[q].empty();) {
        const HEntry top = hq[q].front();
        std::pop_heap(hq[q].begin(), hq[q].end(), hworse);
        hq[q].pop_back();
        State& st = states[top.idx];
        if (st.closed || top.g > st.g || top.g > best_g) continue;
        st.closed = true;
        out.push_back(top.idx);
        ++n;
      }
    }
    if (learned()) {  // learned queue: gather the pool; the caller scores it and calls choose()
      const int L = std::max(16, 2 * B);
      pool.clear();
      while ((int)pool.size() < L && !hq[2].empty()) {
        const HEntry top = hq[2].front();
        std::pop_heap(hq[2].begin(), hq[2].end(), hworse);
        hq[2].pop_back();
        State& st = states[top.idx];
        if (st.closed || top.g > st.g || top.g > best_g) continue;
        if (std::find(pool.begin(), pool.end(), top.idx) != pool.end()) continue;
        pool.push_back(top.idx);
      }
    }
    if (out.empty() && heap.empty() && pool.empty()) done = true;
  }
  // learned queue: expand the B pool states of smallest g + h_cnn; the rest go back
  void choose(int B, std::vector<int>& out) {
    std::vector<int> live;
    for (int idx : pool)
      if (!states[idx].closed) live.push_back(idx);
    const bool by_depth = dive();
    std::sort(live.begin(), live.end(), [this, by_depth](int a, int b) {
      const size_t da = states[a].depth, db = states[b].depth;
      if (by_depth && da != db) return da > db;  // deepest first, as the pool
      const double fa = (double)states[a].g + states[a].h_cnn, fb = (double)states[b].g + states[b].h_cnn;
      if (fa != fb) return fa < fb;
      if (da != db) return da > db;
      return a < b;
    });
    for (size_t k = 0; k < live.size(); ++k) {
      if ((int)k < B) {
        states[live[k]].closed = true;
        out.push_back(live[k]);
      } else {
        hq[2].push_back(HEntry{hval(2, live[k]), states[live[k]].g, live[k]});
        std::push_heap(hq[2].begin(), hq[2].end(), hworse);
      }
    }
    pool.clear();
  }
  // learned queue: the expansion record of state `pidx` from its children's records
  void record_expansion(int pidx, const perch_obj* hyps, const perch_cost* recs, long long n) {
    ExpansionRecord er;
    er.types = remaining(key_of(pidx));
    const size_t nt = er.types.size();
    er.top.assign(nt * T, perch_obj{0xffff, 0, 0, 0});
    er.best.assign(nt, kInf);
    std::vector<std::vector<std::pair<int64_t, long long>>> by(nt);
    for (long long h = 0; h < n; ++h) {
      if (recs[h].flags & kNoCost) {
        bad_record = true;
        continue;
      }
      if (recs[h].viol > 0) continue;
      const size_t t = std::lower_bound(er.types.begin(), er.types.end(), (int)hyps[h].mesh) - er.types.begin();
      if (t >= nt) continue;
      by[t].push_back({(int64_t)recs[h].djr + recs[h].djo + recs[h].resid, h});
    }
    for (size_t t = 0; t < nt; ++t) {
      const size_t k = std::min<size_t>(T, by[t].size());
      std::partial_sort(by[t].begin(), by[t].begin() + k, by[t].end());
      for (size_t j = 0; j < k; ++j) er.top[t * T + j] = hyps[by[t][j].second];
      if (k) er.best[t] = by[t][0].first;
    }
    for (int m : remaining_multiset(key_of(pidx))) {
      const size_t t = std::lower_bound(er.types.begin(), er.types.end(), m) - er.types.begin();
      er.total += (t < nt && er.best[t] != kInf) ? er.best[t] : (int64_t)1 << 40;
    }
    states[pidx].exp = (int)exps.size();
    exps.push_back(std::move(er));
  }
  std::vector<int> remaining_multiset(const Key& key) const {
    std::vector<int> rem = multiset;
    for (uint64_t k : key) {
      auto it = std::find(rem.begin(), rem.end(), (int)(k >> 48));
      if (it != rem.end()) rem.erase(it);
    }
    std::sort(rem.begin(), rem.end());
    return rem;
  }
  // pop up to B expandable states; marks the search done when none is left
  void pop(int B, std::vector<int>& out) {
    out.clear();
    if (diving && dive_next >= 0) {  // greedy completion: its one state this round
      dive_from = dive_next;
      dive_next = -1;
      states[dive_from].closed = true;
      out.push_back(dive_from);
      return;
    }
    if (focal()) {
      pop_focal(B, out);
      return;
    }
    auto cmp = [this](const OpenEntry& a, const OpenEntry& b) { return worse(a, b); };
    while (!heap.empty() && (int)out.size() < B) {
      const OpenEntry top = heap.front();
      if (top.g > best_g) break;
      std::pop_heap(heap.begin(), heap.end(), cmp);
      heap.pop_back();
      State& s = states[top.idx];
      if (s.closed || top.g > s.g) continue;  // stale entry
      s.closed = true;
      out.push_back(top.idx);
    }
    if (out.empty() && (heap.empty() || heap.front().g > best_g)) done = true;
  }
  // distinct unplaced types of a state (the branching of Sec. IV-B)
  std::vector<int> remaining(const Key& key) const {
    std::vector<int> rem = multiset;
    for (uint64_t k : key) {
      auto it = std::find(rem.begin(), rem.end(), (int)(k >> 48));
      if (it != rem.end()) rem.erase(it);
    }
    std::sort(rem.begin(), rem.end());
    rem.erase(std::unique(rem.begin(), rem.end()), rem.end());
    return rem;
  }
  // the child idx = pidx + {o}: its free estimate is the parent's total less
  // the cheapest cost of o's type (o itself is valid, so that type has one)
  void set_parent(int idx, int pidx, const perch_obj& o) {
    State& s = states[idx];
    s.parent = pidx;
    const ExpansionRecord& er = exps[states[pidx].exp];
    const size_t t = std::lower_bound(er.types.begin(), er.types.end(), (int)o.mesh) - er.types.begin();
    s.h_free = er.total - ((t < er.types.size() && er.best[t] != kInf) ? er.best[t] : (int64_t)1 << 40);
    s.h_cnn = -1.0;  // candidates changed: score again
  }
  // greedy completion: child idx of the state it expands; keep the cheapest
  // (ties: the smallest key)
  void dive_offer(int idx) {
    const int64_t g = states[idx].g;
    if (dive_pick < 0 || g < dive_pick_g || (g == dive_pick_g && key_of(idx) < key_of(dive_pick))) {
      dive_pick = idx;
      dive_pick_g = g;
    }
  }
  void absorb(int pidx, const perch_obj& h, const perch_cost& r) {
    if (r.flags & kNoCost) {  // no cost was computed: the search cannot go on
      bad_record = true;
      return;
    }
    if (r.viol > 0) return;  // occludes the parent: not a successor (Eq. (3))
    const int64_t ng = states[pidx].g + (int64_t)r.djr + r.djo + r.resid;
    if (ng > best_g) return;
    const uint64_t o = pack(h);
    const State& ps = states[pidx];
    if (ps.depth + 1 == K) {  // a goal: only its cost and key matter
      if (ng < best_g) {
        best_g = ng;
        best_key = key_of(pidx);
        best_key.insert(std::upper_bound(best_key.begin(), best_key.end(), o), o);
        found_seconds = now;
        found_expansions = expansions;
      } else if (ng == best_g) {
        Key ck = key_of(pidx);
        ck.insert(std::upper_bound(ck.begin(), ck.end(), o), o);
        if (ck < best_key) {
          best_key = std::move(ck);
          found_seconds = now;
          found_expansions = expansions;
        }
      }
      return;
    }
    const uint64_t h0 = ps.hk0 + zobj0(o), h1 = ps.hk1 + zobj1(o);
    const int found =
        index.find(h0, [&](int i) { return states[i].hk1 == h1 && same_set(i, pidx, o); });
    if (found < 0) {
      const int idx = (int)states.size();
      State c;
      c.g = ng;
      c.h_overlap = ps.h_overlap - (int64_t)r.n_vol;
      c.hk0 = h0;
      c.hk1 = h1;
      c.obj = o;
      c.link = pidx;
      c.depth = (uint8_t)(ps.depth + 1);
      states.push_back(c);
      index.insert(h0, idx);
      if (learned()) set_parent(idx, pidx, h);
      add_open(ng, idx);
      if (pidx == dive_from) dive_offer(idx);
    } else {
      State& s = states[found];
      if (ng < s.g) {
        s.g = ng;
        s.closed = false;  // a cheaper way in: reopen
        if (learned() && s.parent != pidx) set_parent(found, pidx, h);
        add_open(ng, found);
      }
      if (pidx == dive_from) dive_offer(found);
    }
  }
};

struct Work {
  int scene_slot;
  int state;
};

// Learned queue: h_cnn of every unscored state in the scenes' pools, one
// batch of crops and one forward pass for all of them.
int score_pools(perch_ctx* ctx, std::vector<SceneSearch>& ss) {
  std::vector<Work> todo;
  int stride = 1;
  for (size_t k = 0; k < ss.size(); ++k)
    for (int idx : ss[k].pool) {
      State& st = ss[k].states[idx];
      if (st.h_cnn >= 0.0) continue;
      if (st.parent < 0) {
        st.h_cnn = 0.0;  // the root: nothing placed, nothing to compare
        continue;
      }
      todo.push_back(Work{(int)k, idx});
      stride = std::max(stride, (int)st.depth);
    }
  const int max_par = std::max(1, 65535 / stride);
  std::vector<perch_obj> parents, hyps;
  std::vector<int32_t> plen, pscene, hparent;
  std::vector<int> hyp_type;  // remaining-type slot of each hypothesis
  std::vector<float> pred;
  for (size_t b0 = 0; b0 < todo.size(); b0 += max_par) {
    const size_t b1 = std::min(todo.size(), b0 + (size_t)max_par);
    parents.assign((b1 - b0) * stride, perch_obj{0, 0, 0, 0});
    plen.assign(b1 - b0, 0);
    pscene.assign(b1 - b0, 0);
    hyps.clear();
    hparent.clear();
    hyp_type.clear();
    std::vector<std::vector<int>> types(b1 - b0);
    for (size_t i = b0; i < b1; ++i) {
      SceneSearch& s = ss[todo[i].scene_slot];
      const State& st = s.states[todo[i].state];
      const size_t w = i - b0;
      const Key key = s.key_of(todo[i].state);
      plen[w] = (int32_t)key.size();
      pscene[w] = s.scene;
      for (size_t j = 0; j < key.size(); ++j) parents[w * stride + j] = unpack(key[j]);
      const ExpansionRecord& er = s.exps[s.states[st.parent].exp];
      types[w] = s.remaining(key);
      for (size_t t = 0; t < types[w].size(); ++t) {
        const size_t et = std::lower_bound(er.types.begin(), er.types.end(), types[w][t]) - er.types.begin();
        if (et >= er.types.size()) continue;
        for (int j = 0; j < s.T; ++j) {
          const perch_obj& o = er.top[et * s.T + j];
          if (o.mesh == 0xffff) break;
          hyps.push_back(o);
          hparent.push_back((int32_t)w);
          hyp_type.push_back((int)t);
        }
      }
    }
    pred.assign(hyps.size(), 0.0f);
    ctx->net_states += (long long)(b1 - b0);
    ctx->net_crops_scored += (long long)hyps.size();
    if (!hyps.empty()) {
      const int rc = net_predict(ctx, ctx->net, parents.data(), stride, plen.data(), pscene.data(),
                                 (int32_t)(b1 - b0), hparent.data(), hyps.data(), (long long)hyps.size(), pred.data());
      if (rc != PERCH_OK) return rc;
    }
    // per state and remaining type: the smallest predicted edge cost
    std::vector<std::vector<double>> best(b1 - b0);
    for (size_t w = 0; w < b1 - b0; ++w) best[w].assign(types[w].size(), 1e7);
    for (size_t h = 0; h < hyps.size(); ++h) {
      const double c = std::max(0.0, std::expm1((double)pred[h]));
      double& b = best[hparent[h]][hyp_type[h]];
      b = std::min(b, c);
    }
    for (size_t i = b0; i < b1; ++i) {
      SceneSearch& s = ss[todo[i].scene_slot];
      State& st = s.states[todo[i].state];
      const size_t w = i - b0;
      double h = 0.0;
      for (int m : s.remaining_multiset(s.key_of(todo[i].state))) {
        const size_t t = std::lower_bound(types[w].begin(), types[w].end(), m) - types[w].begin();
        h += t < types[w].size() ? best[w][t] : 1e7;
      }
      st.h_cnn = h;
    }
  }
  return PERCH_OK;
}

// Run the searches until every one is done or a limit is reached.
int run_searches(perch_ctx* ctx, std::vector<SceneSearch>& ss, int batch_states, double time_limit_s,
                 int64_t max_expansions, int64_t max_hyps_per_launch, bool multi) {
  const auto t0 = Clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(Clock::now() - t0).count(); };
  ctx->net_seconds = ctx->search_eval_seconds = ctx->search_absorb_seconds = ctx->search_host_seconds = 0.0;
  ctx->net_states = ctx->net_crops_scored = 0;
  int stride = 1;
  for (auto& s : ss) stride = std::max(stride, s.K - 1);
  const int B = std::max(1, std::min(batch_states, 65535 / stride));
  const int64_t per_state_max = (int64_t)ctx->nx * ctx->ny * ctx->n_yaw * ctx->n_mesh;
  std::vector<perch_obj> parents, hyps;
  std::vector<int32_t> plen, pscene, pK, hparent;
  std::vector<perch_cost> out;
  std::vector<Work> work;
  std::vector<int> popped;
  std::vector<std::vector<int>> rem, by_scene;  // per work item: remaining types; per scene slot: work items
  std::vector<int> slots;
  int64_t expansions = 0;
  size_t rr = 0;  // round-robin start over scenes
  while (true) {
    const auto tr = Clock::now();
    bool any = false;
    for (auto& s : ss) any |= !s.done;
    if (!any) return PERCH_OK;
    if ((time_limit_s > 0 && elapsed() > time_limit_s) || (max_expansions > 0 && expansions >= max_expansions))
      return PERCH_E_TIMEOUT;
    // gather expansions across scenes, within the launch budgets
    work.clear();
    int64_t budget = max_hyps_per_launch > 0 ? std::max<int64_t>(max_hyps_per_launch, per_state_max)
                                             : (int64_t)B * per_state_max * (int64_t)ss.size();
    std::vector<int> wants(ss.size(), 0);
    bool any_pool = false;
    for (size_t k = 0; k < ss.size() && budget > 0 && (int)work.size() < 65535 / stride; ++k) {
      const size_t si = (rr + k) % ss.size();
      SceneSearch& s = ss[si];
      if (s.done) continue;
      const int want = (int)std::max<int64_t>(1, std::min<int64_t>(B, budget / std::max<int64_t>(per_state_max, 1)));
      s.pop(want, popped);
      if (s.done) s.seconds = elapsed();
      for (int idx : popped) {
        work.push_back(Work{(int)si, idx});
        budget -= per_state_max;
      }
      wants[si] = want;
      any_pool |= !s.pool.empty();
    }
    if (any_pool) {  // learned queue: score the pools, then take each scene's best
      if (!ctx->net) return ctx->fail(PERCH_E_STATE, "search: heuristic bits 2 and 3 need perch_set_heuristic_net");
      const auto ts = Clock::now();
      const int rc = score_pools(ctx, ss);
      ctx->net_seconds += std::chrono::duration<double>(Clock::now() - ts).count();
      if (rc != PERCH_OK) return rc;
      for (size_t si = 0; si < ss.size(); ++si) {
        if (ss[si].pool.empty()) continue;
        popped.clear();
        ss[si].choose(std::max(1, wants[si]), popped);
        for (int idx : popped) {
          if ((int)work.size() >= 65535 / stride) {  // no room this launch: back into the open set
            ss[si].states[idx].closed = false;
            ss[si].add_open(ss[si].states[idx].g, idx);
            continue;
          }
          work.push_back(Work{(int)si, idx});
        }
      }
    }
    rr = (rr + 1) % ss.size();
    if (work.empty()) continue;
    parents.assign(work.size() * stride, perch_obj{0, 0, 0, 0});
    plen.assign(work.size(), 0);
    pscene.assign(work.size(), 0);
    pK.assign(work.size(), 1);
    // every pose of every remaining type, per expanded state: offsets first,
    // then the (independent) per-state fills in parallel
    std::vector<size_t> hbeg(work.size() + 1, 0);
    rem.resize(work.size());
    const size_t positions = (size_t)ctx->nx * ctx->ny;
    for (size_t w = 0; w < work.size(); ++w) {
      const SceneSearch& s = ss[work[w].scene_slot];
      const Key key = s.key_of(work[w].state);
      plen[w] = (int32_t)key.size();
      pscene[w] = s.scene;
      pK[w] = s.K;
      for (size_t j = 0; j < key.size(); ++j) parents[w * stride + j] = unpack(key[j]);
      rem[w] = s.remaining(key);
      size_t n = 0;
      for (int m : rem[w]) n += positions * ctx->search_yaws[m].size();
      hbeg[w + 1] = hbeg[w] + n;
    }
    hyps.resize(hbeg[work.size()]);
    hparent.resize(hbeg[work.size()]);
    const int nx = ctx->nx, ny = ctx->ny;
#pragma omp parallel for schedule(dynamic, 1) if (hbeg[work.size()] >= kParallelMin)
    for (long long w = 0; w < (long long)work.size(); ++w) {
      size_t h = hbeg[w];
      for (int m : rem[w])
        for (int ix = 0; ix < nx; ++ix)
          for (int iy = 0; iy < ny; ++iy)
            for (int k : ctx->search_yaws[m]) {
              hyps[h] = perch_obj{(uint16_t)m, (uint16_t)k, (int16_t)ix, (int16_t)iy};
              hparent[h] = (int32_t)w;
              ++h;
            }
    }
    out.resize(hyps.size());
    const auto te = Clock::now();
    ctx->search_host_seconds += std::chrono::duration<double>(te - tr).count();
    const int rc = multi ? perch_eval_successors_multi(ctx, parents.data(), stride, plen.data(), pscene.data(),
                                                       pK.data(), (int32_t)work.size(), hparent.data(),
                                                       hyps.data(), (int64_t)hyps.size(), out.data())
                         : perch_eval_successors(ctx, parents.data(), stride, plen.data(), (int32_t)work.size(),
                                                 hparent.data(), hyps.data(), (int64_t)hyps.size(), ss[0].K,
                                                 out.data());
    if (rc != PERCH_OK) return rc;
    const auto ta = Clock::now();
    ctx->search_eval_seconds += std::chrono::duration<double>(ta - te).count();
    expansions += (int64_t)work.size();
    // Scenes share nothing, so each scene's expansions and records are taken
    // by one thread, in batch order: per scene the same sequence as a single
    // thread taking the whole batch (results do not depend on the threads).
    for (auto& v : by_scene) v.clear();
    by_scene.resize(ss.size());
    slots.clear();
    for (size_t w = 0; w < work.size(); ++w) {
      std::vector<int>& v = by_scene[work[w].scene_slot];
      if (v.empty()) slots.push_back(work[w].scene_slot);
      v.push_back((int)w);
    }
    std::atomic<bool> failed{false};
    const double now = elapsed();
    for (int si : slots) ss[si].now = now;
    auto absorb_scene = [&](int si) {
      try {
        SceneSearch& s = ss[si];
        for (int w : by_scene[si]) {
          s.expansions++;
          if (s.learned())
            s.record_expansion(work[w].state, hyps.data() + hbeg[w], out.data() + hbeg[w],
                               (long long)(hbeg[w + 1] - hbeg[w]));
        }
        for (int w : by_scene[si])
          for (size_t h = hbeg[w]; h < hbeg[w + 1]; ++h) {
            s.successors++;
            s.absorb(work[w].state, hyps[h], out[h]);
          }
        s.end_round();
      } catch (...) {
        failed = true;
      }
    };
#pragma omp parallel for schedule(dynamic, 1) if (slots.size() > 1 && hyps.size() >= kParallelMin)
    for (long long i = 0; i < (long long)slots.size(); ++i) absorb_scene(slots[i]);
    if (failed) return ctx->fail(PERCH_E_OOM, "search: out of host memory while absorbing records");
    for (int si : slots)
      if (ss[si].bad_record)
        return ctx->fail(PERCH_E_DEVICE, "search: an evaluation record carries no cost (flags bit 30 or 31)");
    ctx->search_absorb_seconds += std::chrono::duration<double>(Clock::now() - ta).count();
  }
}

void fill_result(const SceneSearch& s, int status, perch_result* res) {
  std::memset(res, 0, sizeof *res);
  res->cost = -1;
  res->expansions = s.expansions;
  res->successors = s.successors;
  res->seconds = s.seconds;
  res->found_seconds = s.found_seconds;
  res->found_expansions = s.found_expansions;
  if (s.best_g != kInf) {
    res->cost = s.best_g;
    res->n_objs = (int32_t)s.best_key.size();
    for (size_t j = 0; j < s.best_key.size(); ++j) res->objs[j] = unpack(s.best_key[j]);
  }
  // w = 1: optimal; w > 1: within w times the optimum (Theorem 2)
  res->proven_optimal = (status == PERCH_OK && s.done && s.best_g != kInf && s.w <= 1.0) ? 1 : 0;
}

int check_params(perch_ctx* ctx, const perch_search_params* prm) {
  if (!prm || prm->K < 1 || prm->K > 16 || !prm->mesh_multiset || prm->batch_states < 1)
    return ctx->fail(PERCH_E_ARG, "search: bad parameters");
  if (!(prm->w >= 1.0f)) return ctx->fail(PERCH_E_ARG, "search: w must be >= 1");
  if (prm->heuristics & ~31) return ctx->fail(PERCH_E_ARG, "search: unknown heuristic bits %d", prm->heuristics);
  if ((prm->heuristics & 12) == 12) return ctx->fail(PERCH_E_ARG, "search: heuristic bits 2 and 3 exclude each other");
  if ((prm->heuristics & 12) && !ctx->net)
    return ctx->fail(PERCH_E_STATE, "search: heuristic bits 2 and 3 need perch_set_heuristic_net");
  for (int i = 0; i < prm->K; ++i)
    if (prm->mesh_multiset[i] >= ctx->n_mesh) return ctx->fail(PERCH_E_ARG, "search: mesh %d out of range", i);
  return PERCH_OK;
}

}  // namespace

extern "C" int perch_search_times(perch_ctx* ctx, double* eval_seconds, double* absorb_seconds,
                                  double* select_seconds) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (eval_seconds) *eval_seconds = ctx->search_eval_seconds;
  if (absorb_seconds) *absorb_seconds = ctx->search_absorb_seconds;
  if (select_seconds) *select_seconds = ctx->search_host_seconds;
  return PERCH_OK;
}

extern "C" int perch_search_stats(perch_ctx* ctx, double* learned_seconds, int64_t* learned_states,
                                  int64_t* learned_crops) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (learned_seconds) *learned_seconds = ctx->net_seconds;
  if (learned_states) *learned_states = ctx->net_states;
  if (learned_crops) *learned_crops = ctx->net_crops_scored;
  return PERCH_OK;
}

extern "C" int perch_search(perch_ctx* ctx, const perch_search_params* prm, perch_result* res) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (!res) return ctx->fail(PERCH_E_ARG, "search: null result");
  int rc = check_params(ctx, prm);
  if (rc) return rc;
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  std::vector<SceneSearch> ss(1);
  ss[0].init(0, prm->K, prm->mesh_multiset, prm->w, prm->heuristics, ctx->scenes.empty() ? 0 : ctx->scenes[0].idx.n);
  ss[0].T = ctx->net_candidates;
  const auto t0 = Clock::now();
  const int status = run_searches(ctx, ss, prm->batch_states, prm->time_limit_s, prm->max_expansions, 0, false);
  if (status != PERCH_OK && status != PERCH_E_TIMEOUT) return status;
  ss[0].seconds = std::chrono::duration<double>(Clock::now() - t0).count();
  fill_result(ss[0], status, res);
  if (status == PERCH_E_TIMEOUT) return ctx->fail(PERCH_E_TIMEOUT, "search limit reached; best so far returned");
  if (ss[0].best_g == kInf) return ctx->fail(PERCH_E_RANGE, "no valid complete scene exists in the tree");
  return PERCH_OK;
}

extern "C" int perch_search_multi(perch_ctx* ctx, int32_t n_scenes, const int32_t* scenes,
                                  const perch_search_params* params, int64_t max_hyps_per_launch,
                                  perch_result* results) {
  if (!ctx) return PERCH_E_ARG;
  ctx->err.clear();
  if (n_scenes < 1 || !scenes || !params || !results) return ctx->fail(PERCH_E_ARG, "search: bad arguments");
  if (!ctx->has_obs) return ctx->fail(PERCH_E_STATE, "set an observation first");
  std::vector<SceneSearch> ss(n_scenes);
  for (int i = 0; i < n_scenes; ++i) {
    int rc = check_params(ctx, &params[i]);
    if (rc) return rc;
    if (scenes[i] < 0 || scenes[i] >= (int)ctx->scenes.size())
      return ctx->fail(PERCH_E_ARG, "search %d: scene %d not set", i, scenes[i]);
    ss[i].init(scenes[i], params[i].K, params[i].mesh_multiset, params[i].w, params[i].heuristics,
               ctx->scenes[scenes[i]].idx.n);
    ss[i].T = ctx->net_candidates;
  }
  double tl = 0.0;
  int64_t me = 0;
  int B = 1;
  for (int i = 0; i < n_scenes; ++i) {
    tl = std::max(tl, params[i].time_limit_s);
    me = std::max(me, params[i].max_expansions);
    B = std::max(B, params[i].batch_states);
  }
  const int status = run_searches(ctx, ss, B, tl, me, std::max<int64_t>(max_hyps_per_launch, 1), true);
  if (status != PERCH_OK && status != PERCH_E_TIMEOUT) return status;
  for (int i = 0; i < n_scenes; ++i) fill_result(ss[i], status, &results[i]);
  if (status == PERCH_E_TIMEOUT) return ctx->fail(PERCH_E_TIMEOUT, "search limit reached; best so far returned");
  return PERCH_OK;
}
