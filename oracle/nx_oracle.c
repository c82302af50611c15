/*
 * FP64 CPU oracle for the NXgraph update sweep (Chi et al., "NXgraph: An
 * Efficient Graph Processing System on a Single Machine", arXiv 1510.06916).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this code; the CUDA path never links
 * it and shares no code with it.
 *
 * It computes the plain definitions that the DSSS sweeps reach (the sweeps
 * only reorder the same sums, min-reductions and synchronous updates,
 * Section II-B), with its own CSR built by counting sort, in double precision:
 *
 *   PageRank family (the paper names PageRank as its main task, Section IV,
 *   without a formula; this is the standard damped form with dangling mass):
 *     p_uv  = 1/outdeg(u)                    (unweighted; every duplicate edge
 *                                             and self-loop counts)
 *           = w_uv / W_u, W_u = sum_v w_uv   (weighted)
 *     Dm    = sum over dangling u (no out-edge) of r_u
 *     r'_v  = (1-alpha) t_v + alpha ( sum_{u->v} p_uv r_u + Dm s_v )
 *     with t = teleport (1/n if not given) and s = t (dangling spread by the
 *     teleport, personalized PageRank) or s = 1/n (uniform spread).
 *   BFS (Algorithms 2-4): depth(root) = 0, others infinity (0xFFFFFFFF);
 *     depth(v) = min over in-edges of depth(u) + 1 — here by a FIFO queue.
 *   WCC: label(v) = the smallest vertex id in v's weakly connected component
 *     (edges taken in both directions, Section II-A) — here by union-find.
 *   SCC: label(v) = the smallest vertex id in v's strongly connected component
 *     (Section IV-D) — here by Tarjan's depth-first search.
 *   Weighted-PageRank adjoint: lambda^0 = g, lambda' = M^T lambda + g with
 *     (M^T lambda)_u = alpha ( sum_v p_uv lambda_v + d_u (sum_v lambda_v)/n ),
 *     dL/dt = (1-alpha) lambda,
 *     dL/dw_uv = alpha r_u / W_u * (lambda_v - sum_v' p_uv' lambda_v').
 *
 * Every function returns 0 on success and -1 on bad arguments or allocation
 * failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_INF 0xFFFFFFFFu

/* In-edge CSR by destination: off[n+1], nbr[m] (sources), eid[m] (input edge
 * index, built only when asked for), by a counting sort that keeps input order
 * within a vertex. */
typedef struct {
  uint64_t* off;
  uint32_t* nbr;
  uint64_t* eid;
} orc_csr;

static void csr_free(orc_csr* c) {
  free(c->off);
  free(c->nbr);
  free(c->eid);
  c->off = NULL;
  c->nbr = NULL;
  c->eid = NULL;
}

/* key[e] picks the bucket (dst for in-CSR, src for out-CSR); val[e] is stored. */
static int csr_build(uint32_t n, uint64_t m, const uint32_t* key, const uint32_t* val,
                     int with_eid, orc_csr* c) {
  c->off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  c->nbr = (uint32_t*)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
  c->eid = with_eid ? (uint64_t*)malloc((size_t)(m ? m : 1) * sizeof(uint64_t)) : NULL;
  uint64_t* fill = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!c->off || !c->nbr || (with_eid && !c->eid) || !fill) {
    free(fill);
    csr_free(c);
    return -1;
  }
  for (uint64_t e = 0; e < m; ++e) c->off[key[e] + 1]++;
  for (uint32_t v = 0; v < n; ++v) c->off[v + 1] += c->off[v];
  memcpy(fill, c->off, ((size_t)n + 1) * sizeof(uint64_t));
  for (uint64_t e = 0; e < m; ++e) {
    uint64_t k = fill[key[e]]++;
    c->nbr[k] = val[e];
    if (c->eid) c->eid[k] = e;
  }
  free(fill);
  return 0;
}

static int check_edges(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst) {
  if (n == 0) return -1;
  for (uint64_t e = 0; e < m; ++e)
    if (src[e] >= n || dst[e] >= n) return -1;
  return 0;
}

/* Out-weight per source: W_u = number of out-edges (w == NULL) or sum of w. */
static double* out_weight(uint32_t n, uint64_t m, const uint32_t* src, const double* w) {
  double* W = (double*)calloc(n, sizeof(double));
  if (!W) return NULL;
  for (uint64_t e = 0; e < m; ++e) W[src[e]] += w ? w[e] : 1.0;
  return W;
}

/* One synchronous PageRank-family step r -> nx (the definition above). */
static void pr_step(uint32_t n, const orc_csr* in, const double* w, const double* W, double alpha,
                    const double* tele, int dangling_by_tele, const double* r, double* nx) {
  double dm = 0.0;
  for (uint32_t u = 0; u < n; ++u)
    if (W[u] == 0.0) dm += r[u];
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; ++v) {
    double s = 0.0;
    for (uint64_t k = in->off[v]; k < in->off[v + 1]; ++k) {
      uint32_t u = in->nbr[k];
      double p = (w ? w[in->eid[k]] : 1.0) / W[u];
      s += p * r[u];
    }
    double t = tele ? tele[v] : 1.0 / (double)n;
    double spread = dangling_by_tele ? t : 1.0 / (double)n;
    nx[v] = (1.0 - alpha) * t + alpha * (s + dm * spread);
  }
}

/*
 * A prepared PageRank problem: the in-edge CSR and out-weights built once, so
 * that a caller can time the iteration loop alone (the build is not part of
 * an iteration). The arithmetic of each step is pr_step above.
 */
typedef struct {
  uint32_t n;
  uint64_t m;
  orc_csr in;
  double* w; /* copy of the weights (NULL: unweighted) */
  double* W;
} orc_pr_problem;

void orc_pr_release(void* h) {
  orc_pr_problem* p = (orc_pr_problem*)h;
  if (!p) return;
  csr_free(&p->in);
  free(p->w);
  free(p->W);
  free(p);
}

/* Builds the problem for edges src/dst (and weights w, nullable); *out
 * receives the handle (release with orc_pr_release). */
int orc_pr_prepare(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                   const double* w, void** out) {
  *out = NULL;
  if (check_edges(n, m, src, dst)) return -1;
  orc_pr_problem* p = (orc_pr_problem*)calloc(1, sizeof(orc_pr_problem));
  if (!p) return -1;
  p->n = n;
  p->m = m;
  if (csr_build(n, m, dst, src, w != NULL, &p->in)) {
    free(p);
    return -1;
  }
  if (w) {
    p->w = (double*)malloc((size_t)(m ? m : 1) * sizeof(double));
    if (!p->w) {
      orc_pr_release(p);
      return -1;
    }
    memcpy(p->w, w, (size_t)m * sizeof(double));
  }
  p->W = out_weight(n, m, src, w);
  if (!p->W) {
    orc_pr_release(p);
    return -1;
  }
  *out = p;
  return 0;
}

/* `iters` synchronous steps of a prepared problem from r0 (NULL: 1/n). */
int orc_pr_iterate(void* h, double alpha, uint32_t iters, const double* tele,
                   int dangling_by_tele, const double* r0, double* r_out) {
  orc_pr_problem* p = (orc_pr_problem*)h;
  if (!p) return -1;
  const uint32_t n = p->n;
  double* a = (double*)malloc((size_t)n * sizeof(double));
  double* b = (double*)malloc((size_t)n * sizeof(double));
  if (!a || !b) {
    free(a);
    free(b);
    return -1;
  }
  for (uint32_t v = 0; v < n; ++v) a[v] = r0 ? r0[v] : 1.0 / (double)n;
  for (uint32_t it = 0; it < iters; ++it) {
    pr_step(n, &p->in, p->w, p->W, alpha, tele, dangling_by_tele, a, b);
    double* t = a;
    a = b;
    b = t;
  }
  memcpy(r_out, a, (size_t)n * sizeof(double));
  free(a);
  free(b);
  return 0;
}

/*
 * PageRank / personalized PageRank / weighted PageRank, `iters` synchronous
 * steps from r0 (NULL: uniform 1/n). w may be NULL (unweighted); tele may be
 * NULL (uniform teleport 1/n). Result in r_out[n].
 */
int orc_pagerank(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                 const double* w, double alpha, uint32_t iters, const double* tele,
                 int dangling_by_tele, const double* r0, double* r_out) {
  void* h = NULL;
  if (orc_pr_prepare(n, m, src, dst, w, &h)) return -1;
  int rc = orc_pr_iterate(h, alpha, iters, tele, dangling_by_tele, r0, r_out);
  orc_pr_release(h);
  return rc;
}

/* BFS depths from `root` over directed edges (Algorithms 2-4). */
int orc_bfs(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint32_t root,
            uint32_t* depth) {
  if (check_edges(n, m, src, dst) || root >= n) return -1;
  orc_csr out;
  if (csr_build(n, m, src, dst, 0, &out)) return -1;
  uint32_t* queue = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  if (!queue) {
    csr_free(&out);
    return -1;
  }
  for (uint32_t v = 0; v < n; ++v) depth[v] = ORC_INF;
  depth[root] = 0;
  uint64_t head = 0, tail = 0;
  queue[tail++] = root;
  while (head < tail) {
    uint32_t u = queue[head++];
    for (uint64_t k = out.off[u]; k < out.off[u + 1]; ++k) {
      uint32_t v = out.nbr[k];
      if (depth[v] == ORC_INF) {
        depth[v] = depth[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  csr_free(&out);
  return 0;
}

static uint32_t uf_find(uint32_t* parent, uint32_t x) {
  uint32_t r = x;
  while (parent[r] != r) r = parent[r];
  while (parent[x] != r) {
    uint32_t nx = parent[x];
    parent[x] = r;
    x = nx;
  }
  return r;
}

/* WCC labels: the minimum vertex id of each weakly connected component. The
 * smaller root always becomes the parent, so every root is its set's minimum. */
int orc_wcc(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint32_t* label) {
  if (check_edges(n, m, src, dst)) return -1;
  for (uint32_t v = 0; v < n; ++v) label[v] = v;
  for (uint64_t e = 0; e < m; ++e) {
    uint32_t a = uf_find(label, src[e]);
    uint32_t b = uf_find(label, dst[e]);
    if (a < b)
      label[b] = a;
    else if (b < a)
      label[a] = b;
  }
  for (uint32_t v = 0; v < n; ++v) label[v] = uf_find(label, v);
  return 0;
}

/*
 * SCC labels (Section IV-D names strongly connected components among its
 * tasks without giving an algorithm): label(v) = the smallest vertex id of the
 * strongly connected component holding v, u and v sharing a component when
 * each reaches the other along directed edges. Computed by Tarjan's algorithm
 * (Tarjan 1972, "Depth-first search and linear graph algorithms"), written
 * with an explicit stack instead of recursion: a vertex is the root of a
 * component when no vertex reached from it in the depth-first search leads
 * back to a vertex discovered before it; the component is then popped from
 * the stack of visited, unassigned vertices.
 */
int orc_scc(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint32_t* label) {
  if (check_edges(n, m, src, dst)) return -1;
  orc_csr out;
  if (csr_build(n, m, src, dst, 0, &out)) return -1;
  uint32_t* index = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* low = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* stk = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));    /* visited, unassigned */
  uint32_t* cs_v = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));   /* DFS path: vertex    */
  uint64_t* cs_e = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));   /* next out-edge       */
  unsigned char* on = (unsigned char*)calloc(n, 1);
  if (!index || !low || !stk || !cs_v || !cs_e || !on) {
    free(index);
    free(low);
    free(stk);
    free(cs_v);
    free(cs_e);
    free(on);
    csr_free(&out);
    return -1;
  }
  for (uint32_t v = 0; v < n; ++v) index[v] = ORC_INF;
  uint32_t next = 0, sp = 0;
  for (uint32_t r = 0; r < n; ++r) {
    if (index[r] != ORC_INF) continue;
    uint32_t depth = 0;
    cs_v[0] = r;
    cs_e[0] = out.off[r];
    index[r] = low[r] = next++;
    stk[sp++] = r;
    on[r] = 1;
    depth = 1;
    while (depth) {
      const uint32_t u = cs_v[depth - 1];
      if (cs_e[depth - 1] < out.off[u + 1]) {
        const uint32_t v = out.nbr[cs_e[depth - 1]++];
        if (index[v] == ORC_INF) { /* descend */
          index[v] = low[v] = next++;
          stk[sp++] = v;
          on[v] = 1;
          cs_v[depth] = v;
          cs_e[depth] = out.off[v];
          ++depth;
        } else if (on[v] && index[v] < low[u]) {
          low[u] = index[v];
        }
        continue;
      }
      /* all out-edges of u done */
      if (low[u] == index[u]) { /* u roots a component: pop it, label = its min id */
        uint32_t k = sp, mn = ORC_INF;
        do {
          --k;
          if (stk[k] < mn) mn = stk[k];
        } while (stk[k] != u);
        for (uint32_t q = k; q < sp; ++q) {
          label[stk[q]] = mn;
          on[stk[q]] = 0;
        }
        sp = k;
      }
      --depth;
      if (depth) {
        const uint32_t p = cs_v[depth - 1];
        if (low[u] < low[p]) low[p] = low[u];
      }
    }
  }
  free(index);
  free(low);
  free(stk);
  free(cs_v);
  free(cs_e);
  free(on);
  csr_free(&out);
  return 0;
}

/*
 * Weighted-PageRank adjoint. Forward: `fwd_iters` steps from r0 = 1/n with
 * teleport `tele` (NULL: 1/n) and uniform dangling spread. Adjoint:
 * lambda^0 = g, then adj_terms-1 updates lambda' = M^T lambda + g, so lambda
 * holds adj_terms terms of the Neumann series sum_k (M^T)^k g. Outputs (each
 * nullable): r_out[n], lambda_out[n], dw[m] (input edge order), dt[n].
 */
int orc_wpr_adjoint(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                    const double* w, double alpha, uint32_t fwd_iters, uint32_t adj_terms,
                    const double* tele, const double* g, double* r_out, double* lambda_out,
                    double* dw, double* dt) {
  if (check_edges(n, m, src, dst) || !w || !g || adj_terms == 0) return -1;
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* W = out_weight(n, m, src, w);
  double* lam = (double*)malloc((size_t)n * sizeof(double));
  double* nl = (double*)malloc((size_t)n * sizeof(double));
  double* y = (double*)malloc((size_t)n * sizeof(double));
  orc_csr out;
  int bad = !r || !W || !lam || !nl || !y;
  if (!bad) bad = csr_build(n, m, src, dst, 1, &out) != 0;
  if (bad) {
    free(r);
    free(W);
    free(lam);
    free(nl);
    free(y);
    return -1;
  }
  if (orc_pagerank(n, m, src, dst, w, alpha, fwd_iters, tele, 0, NULL, r)) {
    free(r);
    free(W);
    free(lam);
    free(nl);
    free(y);
    csr_free(&out);
    return -1;
  }
  memcpy(lam, g, (size_t)n * sizeof(double));
  for (uint32_t k = 1; k < adj_terms; ++k) {
    double total = 0.0;
    for (uint32_t v = 0; v < n; ++v) total += lam[v];
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t u = 0; u < (int64_t)n; ++u) {
      double s = 0.0;
      for (uint64_t q = out.off[u]; q < out.off[u + 1]; ++q)
        s += (w[out.eid[q]] / W[u]) * lam[out.nbr[q]];
      double dang = (W[u] == 0.0) ? total / (double)n : 0.0;
      nl[u] = alpha * (s + dang) + g[u];
    }
    double* t = lam;
    lam = nl;
    nl = t;
  }
  /* y_u = sum_v p_uv lambda_v */
  for (uint32_t u = 0; u < n; ++u) {
    double s = 0.0;
    for (uint64_t q = out.off[u]; q < out.off[u + 1]; ++q)
      s += (w[out.eid[q]] / W[u]) * lam[out.nbr[q]];
    y[u] = s;
  }
  if (dw)
    for (uint64_t e = 0; e < m; ++e) {
      uint32_t u = src[e], v = dst[e];
      dw[e] = alpha * r[u] / W[u] * (lam[v] - y[u]);
    }
  if (dt)
    for (uint32_t v = 0; v < n; ++v) dt[v] = (1.0 - alpha) * lam[v];
  if (r_out) memcpy(r_out, r, (size_t)n * sizeof(double));
  if (lambda_out) memcpy(lambda_out, lam, (size_t)n * sizeof(double));
  free(r);
  free(W);
  free(lam);
  free(nl);
  free(y);
  csr_free(&out);
  return 0;
}

/* Threads of the parallel loops from now on (k >= 1); the results do not
 * depend on it: every vertex's sum is taken by one thread in edge order. */
void orc_set_threads(int k) {
#ifdef _OPENMP
  if (k >= 1) omp_set_num_threads(k);
#else
  (void)k;
#endif
}
