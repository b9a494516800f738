/*
 * CPU oracle for the frontier-operator graph primitives.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product (the CUDA
 * library and its Python binding) never calls it and shares no code with it.
 *
 * Each routine is the plain textbook definition of what the paper's
 * primitive computes (Sec. 5), single-threaded, written for a reader to check
 * by eye rather than for speed:
 *
 *   or_bfs       FIFO-queue breadth-first search (Sec. 5.1): depth = hop
 *                count from the source, -1 if unreached; parent = the vertex
 *                that first discovered it in queue order, parent[src] = src.
 *   or_sssp      Dijkstra with a binary heap over non-negative integer
 *                weights (Sec. 4.1 "Expressing SSSP", Alg. 1 semantics:
 *                labels start at infinity, label[root] = 0). Distances are
 *                accumulated in 64 bits and stored as uint32, unreachable =
 *                0xFFFFFFFF. pred[v] = the smallest u with an edge (u, v) and
 *                dist[u] + w(u, v) == dist[v]; pred[src] = src; -1 if
 *                unreachable.
 *   or_bc        Brandes' betweenness centrality (Sec. 5.3), unweighted: one
 *                BFS per source counting shortest paths (sigma), then the
 *                dependency pass in reverse BFS order,
 *                delta[v] += sigma[v] / sigma[w] * (1 + delta[w]) for every w
 *                one level below v, and bc[w] += delta[w] for w != s. Sums
 *                over the given sources, with no halving and no scaling.
 *   or_cc        Connected components (Sec. 5.4) by union-find with path
 *                compression; label[v] = smallest vertex id in its component.
 *   or_pagerank  PageRank power iteration in FP64 (Sec. 5.5):
 *                r'[v] = (1-d)/n + d * (sum over edges (u,v) of r[u]/deg(u)
 *                        + D/n), D = sum of r[u] over vertices with deg 0,
 *                starting from r = 1/n, stopping after max_iter iterations or
 *                once sum |r' - r| < tol.
 *
 *
 * Beyond the five primitives (the paper's Sec. 5.5 "Bipartite graphs" and
 * Sec. 7 "neighborhood operations"):
 *
 *   or_neighbor_reduce  for each vertex v of a frontier (or every vertex):
 *                out[v] = the sum, the weighted sum (w(e) * x[u]), the
 *                minimum or the maximum of x[u] over the entries e = (v, u)
 *                of v's row; a vertex without entries gets the operation's
 *                identity (0, +inf -> INT32_MAX, -inf -> INT32_MIN).
 *   or_hits      Kleinberg's hubs and authorities on a bipartite graph
 *                (left vertices [0, n_left) are hubs, the others
 *                authorities): a[r] = sum of h[l] over the hubs l linked
 *                to r, then h[l] = sum of a[r] over the authorities r linked
 *                to l, each vector scaled to unit Euclidean length after
 *                its update; h starts at 1/sqrt(n_left).
 *   or_salsa     SALSA (Lempel and Moran) on the same bipartite graph: the
 *                two random walks' alternating steps, a[r] = sum of
 *                h[l]/deg(l), then h[l] = sum of a[r]/deg(r); h starts
 *                uniform over the hubs that have links.
 *   or_ppr       personalized PageRank (Haveliwala): the PageRank iteration
 *                above with the teleport and the dangling mass sent to the
 *                seed vertices (uniformly) instead of to all vertices.
 *   The three rankings stop after max_iter iterations or once the summed
 *   absolute change of their vectors falls below tol.
 *
 * Graphs are CSR: row_off[n+1] (int32, row_off[0] = 0), col[m] (int32).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- BFS */
int or_bfs(int32_t n, const int32_t *row_off, const int32_t *col, int32_t src,
           int32_t *depth, int32_t *parent) {
  if (n < 1 || src < 0 || src >= n) return -1;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!queue) return -2;
  for (int32_t v = 0; v < n; ++v) {
    depth[v] = -1;
    if (parent) parent[v] = -1;
  }
  int64_t head = 0, tail = 0;
  depth[src] = 0;
  if (parent) parent[src] = src;
  queue[tail++] = src;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
      int32_t v = col[e];
      if (depth[v] == -1) {
        depth[v] = depth[u] + 1;
        if (parent) parent[v] = u;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return 0;
}

/* --------------------------------------------------------------- SSSP */
typedef struct {
  uint64_t key;
  int32_t v;
} heap_item;

static void heap_push(heap_item *h, int64_t *size, uint64_t key, int32_t v) {
  int64_t i = (*size)++;
  h[i].key = key;
  h[i].v = v;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].key <= h[i].key) break;
    heap_item t = h[p];
    h[p] = h[i];
    h[i] = t;
    i = p;
  }
}

static heap_item heap_pop(heap_item *h, int64_t *size) {
  heap_item top = h[0];
  h[0] = h[--(*size)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, s = i;
    if (l < *size && h[l].key < h[s].key) s = l;
    if (r < *size && h[r].key < h[s].key) s = r;
    if (s == i) break;
    heap_item t = h[s];
    h[s] = h[i];
    h[i] = t;
    i = s;
  }
  return top;
}

int or_sssp(int32_t n, const int32_t *row_off, const int32_t *col,
            const uint32_t *w, int32_t src, uint32_t *dist, int32_t *pred) {
  if (n < 1 || src < 0 || src >= n) return -1;
  const uint64_t INF = UINT64_MAX;
  int64_t m = row_off[n];
  uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
  uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
  /* lazy-deletion heap: at most one entry per successful relaxation */
  heap_item *heap = (heap_item *)malloc(sizeof(heap_item) * (size_t)(m + 1));
  if (!d || !done || !heap) {
    free(d); free(done); free(heap);
    return -2;
  }
  for (int32_t v = 0; v < n; ++v) d[v] = INF;
  int64_t hs = 0;
  d[src] = 0;
  heap_push(heap, &hs, 0, src);
  while (hs > 0) {
    heap_item it = heap_pop(heap, &hs);
    int32_t u = it.v;
    if (done[u] || it.key != d[u]) continue;
    done[u] = 1;
    for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
      int32_t v = col[e];
      uint64_t nd = d[u] + (uint64_t)w[e];
      if (nd < d[v]) {
        d[v] = nd;
        heap_push(heap, &hs, nd, v);
      }
    }
  }
  int rc = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (d[v] == INF) {
      dist[v] = 0xFFFFFFFFu;
    } else if (d[v] >= 0xFFFFFFFFull) {
      dist[v] = 0xFFFFFFFFu; /* does not fit the output type */
      rc = -3;
    } else {
      dist[v] = (uint32_t)d[v];
    }
  }
  if (pred) {
    for (int32_t v = 0; v < n; ++v) pred[v] = -1;
    /* smallest u on a shortest-path edge into v; rows are visited in
       increasing u, so the first hit is the smallest */
    for (int32_t u = 0; u < n; ++u) {
      if (d[u] == INF) continue;
      for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
        int32_t v = col[e];
        if (v == src || pred[v] != -1) continue;
        if (d[u] + (uint64_t)w[e] == d[v]) pred[v] = u;
      }
    }
    pred[src] = src;
  }
  free(d);
  free(done);
  free(heap);
  return rc;
}

/* ----------------------------------------------------------------- BC */
int or_bc(int32_t n, const int32_t *row_off, const int32_t *col,
          const int32_t *srcs, int32_t k, double *bc) {
  if (n < 1 || k < 0) return -1;
  for (int32_t i = 0; i < k; ++i)
    if (srcs[i] < 0 || srcs[i] >= n) return -1;
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  double *sigma = (double *)malloc(sizeof(double) * (size_t)n);
  double *delta = (double *)malloc(sizeof(double) * (size_t)n);
  if (!dist || !order || !sigma || !delta) {
    free(dist); free(order); free(sigma); free(delta);
    return -2;
  }
  for (int32_t v = 0; v < n; ++v) bc[v] = 0.0;
  for (int32_t si = 0; si < k; ++si) {
    int32_t s = srcs[si];
    for (int32_t v = 0; v < n; ++v) {
      dist[v] = -1;
      sigma[v] = 0.0;
      delta[v] = 0.0;
    }
    /* forward: BFS order; sigma[w] sums sigma[v] over edges (v, w) with
       dist[w] == dist[v] + 1 */
    int64_t head = 0, tail = 0;
    dist[s] = 0;
    sigma[s] = 1.0;
    order[tail++] = s;
    while (head < tail) {
      int32_t v = order[head++];
      for (int32_t e = row_off[v]; e < row_off[v + 1]; ++e) {
        int32_t w = col[e];
        if (dist[w] < 0) {
          dist[w] = dist[v] + 1;
          order[tail++] = w;
        }
        if (dist[w] == dist[v] + 1) sigma[w] += sigma[v];
      }
    }
    /* backward: reverse BFS order; every w one level below v has its final
       delta when v is processed */
    for (int64_t i = tail - 1; i >= 0; --i) {
      int32_t v = order[i];
      for (int32_t e = row_off[v]; e < row_off[v + 1]; ++e) {
        int32_t w = col[e];
        if (dist[w] == dist[v] + 1)
          delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w]);
      }
      if (v != s) bc[v] += delta[v];
    }
  }
  free(dist);
  free(order);
  free(sigma);
  free(delta);
  return 0;
}

/* ----------------------------------------------------------------- CC */
static int32_t uf_find(int32_t *p, int32_t x) {
  int32_t r = x;
  while (p[r] != r) r = p[r];
  while (p[x] != r) { /* path compression */
    int32_t nx = p[x];
    p[x] = r;
    x = nx;
  }
  return r;
}

int or_cc(int32_t n, const int32_t *row_off, const int32_t *col,
          int32_t *label, int32_t *num_components) {
  if (n < 1) return -1;
  int32_t *p = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!p) return -2;
  for (int32_t v = 0; v < n; ++v) p[v] = v;
  for (int32_t u = 0; u < n; ++u) {
    for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) {
      int32_t a = uf_find(p, u), b = uf_find(p, col[e]);
      if (a == b) continue;
      /* keep the smaller id as the root so the root is the component's
         minimum vertex */
      if (a < b) p[b] = a; else p[a] = b;
    }
  }
  int32_t count = 0;
  for (int32_t v = 0; v < n; ++v) {
    label[v] = uf_find(p, v);
    if (label[v] == v) ++count;
  }
  if (num_components) *num_components = count;
  free(p);
  return 0;
}

/* ----------------------------------------------------------- PageRank */
int or_pagerank(int32_t n, const int32_t *row_off, const int32_t *col,
                double damping, int32_t max_iter, double tol, double *rank,
                int32_t *iters_out) {
  if (n < 1 || max_iter < 0 || !(damping > 0.0 && damping < 1.0)) return -1;
  double *next = (double *)malloc(sizeof(double) * (size_t)n);
  if (!next) return -2;
  for (int32_t v = 0; v < n; ++v) rank[v] = 1.0 / n;
  int32_t it = 0;
  while (it < max_iter) {
    double dangling = 0.0;
    for (int32_t u = 0; u < n; ++u) {
      next[u] = 0.0;
      if (row_off[u + 1] == row_off[u]) dangling += rank[u];
    }
    for (int32_t u = 0; u < n; ++u) {
      int32_t deg = row_off[u + 1] - row_off[u];
      for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e)
        next[col[e]] += rank[u] / deg;
    }
    double diff = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      double r = (1.0 - damping) / n + damping * (next[v] + dangling / n);
      diff += r > rank[v] ? r - rank[v] : rank[v] - r;
      rank[v] = r;
    }
    ++it;
    if (diff < tol) break;
  }
  if (iters_out) *iters_out = it;
  free(next);
  return 0;
}

/* ------------------------------------------------- neighbourhood reduce */
enum { OR_REDUCE_SUM = 0, OR_REDUCE_WSUM = 1, OR_REDUCE_MIN = 2, OR_REDUCE_MAX = 3 };

int or_neighbor_reduce(int32_t n, const int32_t *row_off, const int32_t *col,
                       const uint32_t *w, int32_t op, const int32_t *frontier, int32_t q,
                       const void *x, void *out) {
  if (n < 1 || op < OR_REDUCE_SUM || op > OR_REDUCE_MAX) return -1;
  if (op == OR_REDUCE_WSUM && !w) return -1;
  const int32_t count = frontier ? q : n;
  for (int32_t i = 0; i < count; ++i) {
    const int32_t v = frontier ? frontier[i] : i;
    if (v < 0 || v >= n) return -1;
    if (op == OR_REDUCE_SUM || op == OR_REDUCE_WSUM) {
      const double *xd = (const double *)x;
      double acc = 0.0;
      for (int32_t e = row_off[v]; e < row_off[v + 1]; ++e)
        acc += (op == OR_REDUCE_WSUM ? (double)w[e] : 1.0) * xd[col[e]];
      ((double *)out)[v] = acc;
    } else {
      const int32_t *xi = (const int32_t *)x;
      int32_t acc = op == OR_REDUCE_MIN ? INT32_MAX : INT32_MIN;
      for (int32_t e = row_off[v]; e < row_off[v + 1]; ++e) {
        const int32_t t = xi[col[e]];
        if (op == OR_REDUCE_MIN ? t < acc : t > acc) acc = t;
      }
      ((int32_t *)out)[v] = acc;
    }
  }
  return 0;
}

/* ---------------------------------------------- bipartite node ranking */
/* Every entry must join a hub (< n_left) and an authority (>= n_left). */
static int bipartite_ok(int32_t n, int32_t n_left, const int32_t *row_off, const int32_t *col) {
  if (n < 1 || n_left < 0 || n_left > n) return 0;
  for (int32_t v = 0; v < n; ++v)
    for (int32_t e = row_off[v]; e < row_off[v + 1]; ++e)
      if ((v < n_left) == (col[e] < n_left)) return 0;
  return 1;
}

static void scale_unit(double *x, int32_t lo, int32_t hi) {
  double ss = 0.0;
  for (int32_t i = lo; i < hi; ++i) ss += x[i] * x[i];
  if (ss > 0.0) {
    const double inv = 1.0 / sqrt(ss);
    for (int32_t i = lo; i < hi; ++i) x[i] *= inv;
  }
}

int or_hits(int32_t n, int32_t n_left, const int32_t *row_off, const int32_t *col,
            int32_t max_iter, double tol, double *score, int32_t *iters_out) {
  if (max_iter < 0 || !bipartite_ok(n, n_left, row_off, col)) return -1;
  double *next = (double *)malloc(sizeof(double) * (size_t)n);
  if (!next) return -2;
  /* score holds h on [0, n_left) and a on [n_left, n) */
  for (int32_t v = 0; v < n; ++v) score[v] = v < n_left ? 1.0 / sqrt((double)n_left) : 0.0;
  int32_t it = 0;
  while (it < max_iter) {
    for (int32_t r = n_left; r < n; ++r) {  /* authorities from hubs */
      double acc = 0.0;
      for (int32_t e = row_off[r]; e < row_off[r + 1]; ++e) acc += score[col[e]];
      next[r] = acc;
    }
    scale_unit(next, n_left, n);
    for (int32_t l = 0; l < n_left; ++l) {  /* hubs from the new authorities */
      double acc = 0.0;
      for (int32_t e = row_off[l]; e < row_off[l + 1]; ++e) acc += next[col[e]];
      next[l] = acc;
    }
    scale_unit(next, 0, n_left);
    double delta = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      delta += fabs(next[v] - score[v]);
      score[v] = next[v];
    }
    ++it;
    if (delta < tol) break;
  }
  free(next);
  if (iters_out) *iters_out = it;
  return 0;
}

int or_salsa(int32_t n, int32_t n_left, const int32_t *row_off, const int32_t *col,
             int32_t max_iter, double tol, double *score, int32_t *iters_out) {
  if (max_iter < 0 || !bipartite_ok(n, n_left, row_off, col)) return -1;
  double *next = (double *)malloc(sizeof(double) * (size_t)n);
  if (!next) return -2;
  int32_t linked = 0;
  for (int32_t l = 0; l < n_left; ++l) linked += row_off[l + 1] > row_off[l];
  for (int32_t v = 0; v < n; ++v)
    score[v] = (v < n_left && row_off[v + 1] > row_off[v]) ? 1.0 / linked : 0.0;
  int32_t it = 0;
  while (it < max_iter) {
    for (int32_t r = n_left; r < n; ++r) {  /* authority step */
      double acc = 0.0;
      for (int32_t e = row_off[r]; e < row_off[r + 1]; ++e) {
        const int32_t l = col[e];
        acc += score[l] / (row_off[l + 1] - row_off[l]);
      }
      next[r] = acc;
    }
    for (int32_t l = 0; l < n_left; ++l) {  /* hub step from the new authorities */
      double acc = 0.0;
      for (int32_t e = row_off[l]; e < row_off[l + 1]; ++e) {
        const int32_t r = col[e];
        acc += next[r] / (row_off[r + 1] - row_off[r]);
      }
      next[l] = acc;
    }
    double delta = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      delta += fabs(next[v] - score[v]);
      score[v] = next[v];
    }
    ++it;
    if (delta < tol) break;
  }
  free(next);
  if (iters_out) *iters_out = it;
  return 0;
}

int or_ppr(int32_t n, const int32_t *row_off, const int32_t *col, const int32_t *seeds,
           int32_t ns, double damping, int32_t max_iter, double tol, double *rank,
           int32_t *iters_out) {
  if (n < 1 || ns < 1 || max_iter < 0 || !(damping > 0.0 && damping < 1.0)) return -1;
  double *tele = (double *)calloc((size_t)n, sizeof(double));
  double *next = (double *)malloc(sizeof(double) * (size_t)n);
  if (!tele || !next) {
    free(tele);
    free(next);
    return -2;
  }
  for (int32_t i = 0; i < ns; ++i) {
    if (seeds[i] < 0 || seeds[i] >= n || tele[seeds[i]] != 0.0) {  /* distinct seeds */
      free(tele);
      free(next);
      return -1;
    }
    tele[seeds[i]] = 1.0 / ns;
  }
  for (int32_t v = 0; v < n; ++v) rank[v] = tele[v];
  int32_t it = 0;
  while (it < max_iter) {
    double dangling = 0.0;
    for (int32_t u = 0; u < n; ++u) {
      next[u] = 0.0;
      if (row_off[u + 1] == row_off[u]) dangling += rank[u];
    }
    for (int32_t u = 0; u < n; ++u) {
      const int32_t deg = row_off[u + 1] - row_off[u];
      for (int32_t e = row_off[u]; e < row_off[u + 1]; ++e) next[col[e]] += rank[u] / deg;
    }
    double delta = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      next[v] = (1.0 - damping) * tele[v] + damping * (next[v] + dangling * tele[v]);
      delta += fabs(next[v] - rank[v]);
      rank[v] = next[v];
    }
    ++it;
    if (delta < tol) break;
  }
  free(tele);
  free(next);
  if (iters_out) *iters_out = it;
  return 0;
}
