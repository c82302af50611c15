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

#define ORC_INF 0xFFFFFFFFu

/* In-edge CSR by destination: off[n+1], nbr[m] (sources), eid[m] (input edge
 * index), built by a counting sort that keeps input order within a vertex. */
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
                     orc_csr* c) {
  c->off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  c->nbr = (uint32_t*)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
  c->eid = (uint64_t*)malloc((size_t)(m ? m : 1) * sizeof(uint64_t));
  uint64_t* fill = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!c->off || !c->nbr || !c->eid || !fill) {
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
    c->eid[k] = e;
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
 * PageRank / personalized PageRank / weighted PageRank, `iters` synchronous
 * steps from r0 (NULL: uniform 1/n). w may be NULL (unweighted); tele may be
 * NULL (uniform teleport 1/n). Result in r_out[n].
 */
int orc_pagerank(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                 const double* w, double alpha, uint32_t iters, const double* tele,
                 int dangling_by_tele, const double* r0, double* r_out) {
  if (check_edges(n, m, src, dst)) return -1;
  orc_csr in;
  if (csr_build(n, m, dst, src, &in)) return -1;
  double* W = out_weight(n, m, src, w);
  double* a = (double*)malloc((size_t)n * sizeof(double));
  double* b = (double*)malloc((size_t)n * sizeof(double));
  if (!W || !a || !b) {
    free(W);
    free(a);
    free(b);
    csr_free(&in);
    return -1;
  }
  for (uint32_t v = 0; v < n; ++v) a[v] = r0 ? r0[v] : 1.0 / (double)n;
  for (uint32_t it = 0; it < iters; ++it) {
    pr_step(n, &in, w, W, alpha, tele, dangling_by_tele, a, b);
    double* t = a;
    a = b;
    b = t;
  }
  memcpy(r_out, a, (size_t)n * sizeof(double));
  free(W);
  free(a);
  free(b);
  csr_free(&in);
  return 0;
}

/* BFS depths from `root` over directed edges (Algorithms 2-4). */
int orc_bfs(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, uint32_t root,
            uint32_t* depth) {
  if (check_edges(n, m, src, dst) || root >= n) return -1;
  orc_csr out;
  if (csr_build(n, m, src, dst, &out)) return -1;
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
  if (!bad) bad = csr_build(n, m, src, dst, &out) != 0;
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
