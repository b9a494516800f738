// Seeded synthetic graph inputs: R-MAT and 2D grid generators, CSR builder,
// symmetric edge weights and source selection.
//
// This module produces INPUTS only. It holds none of the traversal arithmetic
// (BFS, SSSP, BC, CC, PageRank); both the CPU oracle and the CUDA library read
// the CSR arrays it writes.
//
// Every random draw comes from one counter-based generator, gg_hash3(seed,
// stream, index), built from the splitmix64 output finaliser (Steele, Lea and
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
// Because each draw depends only on (seed, stream, index), the output does not
// depend on the number of threads or their schedule.
//
// Graph shapes follow the paper's workloads (Sec. 6, Table 1): a generated
// scale-free R-MAT graph stands in for kron_g500-logn21, and a 2D mesh with
// random edge deletions stands in for the large-diameter rgg/roadnet graphs.
// All graphs are symmetrised (the paper converts every dataset to undirected),
// self-loops are dropped and each row's columns are sorted ascending with
// duplicates removed.

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

inline uint64_t fmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

inline uint64_t hash3(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t h = fmix64(seed + kGolden);
  h = fmix64(h ^ (stream + 2 * kGolden));
  return fmix64(h ^ (idx + 3 * kGolden));
}

// uniform integer in [0, range) from a 64-bit hash (multiply-high)
inline uint64_t mulhi_range(uint64_t h, uint64_t range) {
  return (uint64_t)(((__uint128_t)h * (__uint128_t)range) >> 64);
}

// Stream tags, so that different uses of one seed never share draws.
constexpr uint64_t kStreamRmat = 0x100;   // + level
constexpr uint64_t kStreamPerm = 0x200;
constexpr uint64_t kStreamGridDel = 0x300;
constexpr uint64_t kStreamWeight = 0x400;
constexpr uint64_t kStreamSource = 0x500;
constexpr uint64_t kStreamBipartite = 0x600;  // + level

int num_threads() {
  const char *env = std::getenv("GG_THREADS");
  if (env && std::atoi(env) > 0) return std::atoi(env);
  unsigned hc = std::thread::hardware_concurrency();
  return hc ? (int)std::min(hc, 64u) : 4;
}

template <class F>
void parallel_for(int64_t n, F f) {
  int t = num_threads();
  if (n < 1 << 16 || t == 1) {
    f(0, n);
    return;
  }
  std::vector<std::thread> ths;
  int64_t chunk = (n + t - 1) / t;
  for (int i = 0; i < t; ++i) {
    int64_t b = i * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    ths.emplace_back([=, &f] { f(b, e); });
  }
  for (auto &th : ths) th.join();
}

struct Csr {
  int32_t n = 0;
  int64_t m = 0;
  std::vector<int32_t> row_off;
  std::vector<int32_t> col;
};

// Build a symmetric, self-loop-free, per-row sorted and deduplicated CSR
// from an undirected edge list (each pair inserted in both directions).
Csr build_symmetric_csr(int32_t n, const std::vector<int32_t> &eu,
                        const std::vector<int32_t> &ev) {
  int64_t ne = (int64_t)eu.size();
  std::vector<std::atomic<int64_t>> cnt(n + 1);
  for (int64_t i = 0; i <= n; ++i) cnt[i].store(0, std::memory_order_relaxed);
  parallel_for(ne, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      int32_t u = eu[i], v = ev[i];
      if (u == v) continue;
      cnt[u].fetch_add(1, std::memory_order_relaxed);
      cnt[v].fetch_add(1, std::memory_order_relaxed);
    }
  });
  std::vector<int64_t> off(n + 1);
  int64_t acc = 0;
  for (int32_t i = 0; i < n; ++i) {
    off[i] = acc;
    acc += cnt[i].load(std::memory_order_relaxed);
  }
  off[n] = acc;
  std::vector<std::atomic<int64_t>> pos(n);
  for (int32_t i = 0; i < n; ++i) pos[i].store(off[i], std::memory_order_relaxed);
  std::vector<int32_t> raw(acc);
  parallel_for(ne, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      int32_t u = eu[i], v = ev[i];
      if (u == v) continue;
      raw[pos[u].fetch_add(1, std::memory_order_relaxed)] = v;
      raw[pos[v].fetch_add(1, std::memory_order_relaxed)] = u;
    }
  });
  // per-row sort + unique
  std::vector<int64_t> newdeg(n);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r) {
      int32_t *p = raw.data() + off[r];
      int64_t len = off[r + 1] - off[r];
      std::sort(p, p + len);
      newdeg[r] = std::unique(p, p + len) - p;
    }
  });
  Csr g;
  g.n = n;
  g.row_off.resize((size_t)n + 1);
  int64_t m = 0;
  for (int32_t r = 0; r < n; ++r) {
    g.row_off[r] = (int32_t)m;  // caller checks m <= INT32_MAX
    m += newdeg[r];
  }
  g.m = m;
  if (m > INT32_MAX) {
    g.n = -1;
    return g;
  }
  g.row_off[n] = (int32_t)m;
  g.col.resize(m);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r)
      std::memcpy(g.col.data() + g.row_off[r], raw.data() + off[r],
                  sizeof(int32_t) * newdeg[r]);
  });
  return g;
}

}  // namespace

extern "C" {

uint64_t gg_hash3(uint64_t seed, uint64_t stream, uint64_t idx) {
  return hash3(seed, stream, idx);
}

// Opaque result holder: gg_*_build returns one, gg_csr_copy fills caller
// buffers, gg_csr_free releases it.
void *gg_rmat_build(int32_t scale, int32_t edge_factor, double a, double b,
                    double c, uint64_t seed, int32_t permute, int32_t *n_out,
                    int64_t *m_out, int64_t *raw_edges_out) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return nullptr;
  int32_t n = 1 << scale;
  int64_t ne = (int64_t)n * edge_factor;
  // cumulative quadrant thresholds on a 53-bit integer uniform
  const double two53 = 9007199254740992.0;
  const uint64_t ta = (uint64_t)(a * two53 + 0.5);
  const uint64_t tab = (uint64_t)((a + b) * two53 + 0.5);
  const uint64_t tabc = (uint64_t)((a + b + c) * two53 + 0.5);
  std::vector<int32_t> perm;
  if (permute) {
    // permutation = argsort of per-vertex hash keys (ties broken by id)
    std::vector<uint64_t> key(n);
    perm.resize(n);
    for (int32_t v = 0; v < n; ++v) {
      key[v] = hash3(seed, kStreamPerm, (uint64_t)v);
      perm[v] = v;
    }
    std::sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) {
      return key[x] != key[y] ? key[x] < key[y] : x < y;
    });
  }
  std::vector<int32_t> eu(ne), ev(ne);
  parallel_for(ne, [&](int64_t b0, int64_t e0) {
    for (int64_t i = b0; i < e0; ++i) {
      uint32_t u = 0, v = 0;
      for (int32_t l = 0; l < scale; ++l) {
        uint64_t r = hash3(seed, kStreamRmat + (uint64_t)l, (uint64_t)i) >> 11;
        uint32_t ub, vb;
        if (r < ta) { ub = 0; vb = 0; }
        else if (r < tab) { ub = 0; vb = 1; }
        else if (r < tabc) { ub = 1; vb = 0; }
        else { ub = 1; vb = 1; }
        u = (u << 1) | ub;
        v = (v << 1) | vb;
      }
      if (permute) { u = perm[u]; v = perm[v]; }
      eu[i] = (int32_t)u;
      ev[i] = (int32_t)v;
    }
  });
  Csr *g = new Csr(build_symmetric_csr(n, eu, ev));
  if (g->n < 0) { delete g; return nullptr; }
  *n_out = g->n;
  *m_out = g->m;
  if (raw_edges_out) *raw_edges_out = ne;
  return g;
}

// Bipartite R-MAT: 2^scale_left hub vertices (ids [0, n_left)) and
// 2^scale_right authority vertices (ids [n_left, n)). Edge i draws a
// max(scale_left, scale_right)-level quadrant path like the square R-MAT
// (its own stream tag); its row bits give the hub (the top scale_left of
// them), its column bits the authority (the top scale_right). Every edge
// joins a hub and an authority; the CSR holds both directions, rows sorted
// and deduplicated.
void *gg_rmat_bipartite_build(int32_t scale_left, int32_t scale_right, int32_t edge_factor,
                              double a, double b, double c, uint64_t seed, int32_t *n_out,
                              int32_t *n_left_out, int64_t *m_out) {
  if (scale_left < 0 || scale_right < 0 || scale_left > 29 || scale_right > 29 ||
      edge_factor < 1)
    return nullptr;
  const int32_t levels = std::max(scale_left, scale_right);
  const int64_t n_left = (int64_t)1 << scale_left, n_right = (int64_t)1 << scale_right;
  if (n_left + n_right > INT32_MAX) return nullptr;
  const int32_t n = (int32_t)(n_left + n_right);
  const int64_t ne = (int64_t)edge_factor * std::max(n_left, n_right);
  const double two53 = 9007199254740992.0;
  const uint64_t ta = (uint64_t)(a * two53 + 0.5);
  const uint64_t tab = (uint64_t)((a + b) * two53 + 0.5);
  const uint64_t tabc = (uint64_t)((a + b + c) * two53 + 0.5);
  std::vector<int32_t> eu(ne), ev(ne);
  parallel_for(ne, [&](int64_t b0, int64_t e0) {
    for (int64_t i = b0; i < e0; ++i) {
      uint32_t u = 0, v = 0;
      for (int32_t l = 0; l < levels; ++l) {
        uint64_t r = hash3(seed, kStreamBipartite + (uint64_t)l, (uint64_t)i) >> 11;
        uint32_t ub, vb;
        if (r < ta) { ub = 0; vb = 0; }
        else if (r < tab) { ub = 0; vb = 1; }
        else if (r < tabc) { ub = 1; vb = 0; }
        else { ub = 1; vb = 1; }
        u = (u << 1) | ub;
        v = (v << 1) | vb;
      }
      eu[i] = (int32_t)(u >> (levels - scale_left));
      ev[i] = (int32_t)(n_left + (v >> (levels - scale_right)));
    }
  });
  Csr *g = new Csr(build_symmetric_csr(n, eu, ev));
  if (g->n < 0) { delete g; return nullptr; }
  *n_out = g->n;
  *n_left_out = (int32_t)n_left;
  *m_out = g->m;
  return g;
}

// side x side 4-neighbour grid; vertex (r, c) has id r*side + c. Each
// undirected edge is deleted independently with probability p_del, keyed by
// its index in a canonical order: horizontal edges (r,c)-(r,c+1) first with
// index r*(side-1)+c, then vertical edges (r,c)-(r+1,c) with index
// H + r*side + c, H = side*(side-1).
void *gg_grid_build(int32_t side, double p_del, uint64_t seed, int32_t *n_out,
                    int64_t *m_out, int64_t *kept_undirected_out) {
  if (side < 1 || (int64_t)side * side > INT32_MAX) return nullptr;
  int64_t n = (int64_t)side * side;
  int64_t H = (int64_t)side * (side - 1);
  int64_t total = 2 * H;
  const uint64_t tdel = (uint64_t)(p_del * 9007199254740992.0 + 0.5);
  std::vector<uint8_t> keep(total);
  parallel_for(total, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i)
      keep[i] = (hash3(seed, kStreamGridDel, (uint64_t)i) >> 11) >= tdel;
  });
  std::vector<int32_t> eu, ev;
  eu.reserve(total);
  ev.reserve(total);
  for (int64_t i = 0; i < total; ++i) {
    if (!keep[i]) continue;
    int64_t u, v;
    if (i < H) {
      int64_t r = i / (side - 1), c = i % (side - 1);
      u = r * side + c;
      v = u + 1;
    } else {
      int64_t j = i - H;
      int64_t r = j / side, c = j % side;
      u = r * side + c;
      v = u + side;
    }
    eu.push_back((int32_t)u);
    ev.push_back((int32_t)v);
  }
  Csr *g = new Csr(build_symmetric_csr((int32_t)n, eu, ev));
  *n_out = g->n;
  *m_out = g->m;
  if (kept_undirected_out) *kept_undirected_out = (int64_t)eu.size();
  return g;
}

void gg_csr_copy(void *h, int32_t *row_off, int32_t *col) {
  Csr *g = (Csr *)h;
  std::memcpy(row_off, g->row_off.data(), sizeof(int32_t) * ((size_t)g->n + 1));
  std::memcpy(col, g->col.data(), sizeof(int32_t) * (size_t)g->m);
}

void gg_csr_free(void *h) { delete (Csr *)h; }

// Symmetric weights in [wmin, wmax]: w(u,v) depends only on the unordered
// pair {u, v}, so both directions of an undirected edge carry the same value.
void gg_weights(const int32_t *row_off, const int32_t *col, int32_t n,
                uint64_t seed, uint32_t wmin, uint32_t wmax, uint32_t *w) {
  uint64_t range = (uint64_t)wmax - wmin + 1;
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t u = b; u < e; ++u) {
      for (int64_t k = row_off[u]; k < row_off[u + 1]; ++k) {
        uint64_t v = (uint64_t)col[k];
        uint64_t lo = std::min<uint64_t>(u, v), hi = std::max<uint64_t>(u, v);
        uint64_t key = lo * (uint64_t)n + hi;
        w[k] = wmin + (uint32_t)mulhi_range(hash3(seed, kStreamWeight, key), range);
      }
    }
  });
}

// Draw `count` distinct vertices of non-zero degree: candidate j is
// floor(hash3(seed, SOURCE, j) * n / 2^64); candidates with degree 0 or
// already drawn are skipped. Returns the number drawn (< count only if the
// attempt limit was reached).
int32_t gg_sources(const int32_t *row_off, int32_t n, int32_t count,
                   uint64_t seed, int32_t *out) {
  int32_t got = 0;
  std::vector<uint8_t> taken(n, 0);
  for (uint64_t j = 0; got < count && j < (uint64_t)n * 64 + 1024; ++j) {
    int32_t v = (int32_t)mulhi_range(hash3(seed, kStreamSource, j), (uint64_t)n);
    if (taken[v] || row_off[v + 1] == row_off[v]) continue;
    taken[v] = 1;
    out[got++] = v;
  }
  return got;
}

// Highest-degree vertex, ties to the smallest id.
int32_t gg_max_degree_vertex(const int32_t *row_off, int32_t n) {
  int32_t best = 0;
  int32_t bd = -1;
  for (int32_t v = 0; v < n; ++v) {
    int32_t d = row_off[v + 1] - row_off[v];
    if (d > bd) { bd = d; best = v; }
  }
  return best;
}

}  // extern "C"
