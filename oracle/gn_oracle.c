/*
 * gn_oracle.c -- plain FP64 CPU oracle for Graph Normalization (GN).
 *
 * TEST INFRASTRUCTURE ONLY (see gn_oracle.h).  Sequential C99, no blocking,
 * fusion or reordering: each function is the definition it cites, written out
 * in the paper's x-space notation so that it can be checked against the paper
 * by eye.  Build with -ffp-contract=off so x86 and Arm hosts agree bit for bit.
 */
#include "gn_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Sec. 2 (graph setting): G is a simple undirected graph, A symmetric with a zero
 * diagonal; Def. WRGN: w > 0.  Checks the CSR encoding of exactly that: rows
 * sorted and duplicate-free, no self-loops, every edge present in both
 * directions, weights finite and positive. */
int gno_validate(int n, const int32_t* rp, const int32_t* ci, const double* w) {
  if (n < 0 || !rp) return GNO_ERR_ARG;
  if (rp[0] != 0) return GNO_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return GNO_ERR_ARG;
  for (int e = 0; e < rp[n]; ++e)      /* a malformed encoding is an argument error first */
    if (ci[e] < 0 || ci[e] >= n) return GNO_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = ci[e];
      if (j == i) return GNO_ERR_NOT_SIMPLE;                    /* self-loop */
      if (e > rp[i] && ci[e - 1] >= j) return GNO_ERR_NOT_SIMPLE; /* unsorted or duplicate */
      int found = 0;                                             /* symmetry: i in N(j) */
      for (int f = rp[j]; f < rp[j + 1]; ++f)
        if (ci[f] == i) { found = 1; break; }
      if (!found) return GNO_ERR_NOT_SIMPLE;
    }
  }
  for (int i = 0; i < n; ++i)
    if (!(w[i] > 0.0) || !isfinite(w[i])) return GNO_ERR_WEIGHT;
  return GNO_OK;
}

/* Sec. 6 (gamma-pursuit) and the appendix PyTorch module: gamma rises linearly
 * from gamma0 to gamma1, t = k/(T-1), gamma = t*gamma1 + (1-t)*gamma0.  Past the
 * ramp (k >= T-1) gamma stays at gamma1.  Fixed mode holds gamma1. */
double gno_gamma(const gno_params* p, int k) {
  if (p->gamma_mode == GNO_GAMMA_FIXED || p->ramp_iters <= 1) return p->gamma1;
  int kk = k < p->ramp_iters - 1 ? k : p->ramp_iters - 1;
  double t = (double)kk / (double)(p->ramp_iters - 1);
  return t * p->gamma1 + (1.0 - t) * p->gamma0;
}

/* Def. WRGN: x_i' = x_i / (x_i + gamma * sum_{j in N(i)} (v_j / v_i) x_j), v = sqrt(w).
 * Safe division of the appendix module: the mask is taken on the weighted-state
 * denominator (B y)_i = v_i * (x_i + gamma sum (v_j/v_i) x_j); when it is <= 1e-9
 * the value is set to 0.5 and the event counted. */
void gno_step(int n, const int32_t* rp, const int32_t* ci, const double* v, double gamma,
              const double* x, double* xn, long long* hits) {
  for (int i = 0; i < n; ++i) {
    double nb = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = ci[e];
      nb += (v[j] / v[i]) * x[j];
    }
    double d = x[i] + gamma * nb;
    if (v[i] * d > 1e-9) {
      xn[i] = x[i] / d;
    } else {
      xn[i] = 0.5;
      if (hits) ++*hits;
    }
  }
}

/* Thm. 3 (weighted mass): M_v(y) = sum v_i y_i = sum w_i x_i, the relaxed MWIS objective. */
double gno_objective(int n, const double* w, const double* x) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += w[i] * x[i];
  return s;
}

/* Sec. 3, energy in the weighted state y = v (.) x:
 *   E~(y) = 1/2 y^T (I + gamma A) y - v^T y. */
double gno_energy(int n, const int32_t* rp, const int32_t* ci, const double* w, double gamma,
                  const double* x) {
  double quad = 0.0, lin = 0.0;
  for (int i = 0; i < n; ++i) {
    double vi = sqrt(w[i]);
    double yi = vi * x[i];
    double ay = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = ci[e];
      ay += sqrt(w[j]) * x[j];
    }
    quad += yi * (yi + gamma * ay);
    lin += vi * yi;
  }
  return 0.5 * quad - lin;
}

static int is_check(int k, int check_every, int max_iters) {
  return ((k + 1) % check_every == 0) || (k + 1 == max_iters);
}

/* Iterated WRGN (Def. IGN applied to the WRGN map) with the gamma-pursuit schedule
 * of Sec. 6, followed by the clamp of the appendix module.  Iterations are the
 * absolute indices k = start_iter .. max_iters-1, so a run resumed from a saved
 * state with start_iter = K reproduces the uninterrupted run.
 *
 * Stop test, evaluated after step k when (k+1) % check_every == 0 or k+1 == max_iters:
 *   binary:   every x_i^{k+1} <= theta or >= 1-theta, and gamma_k (1 - theta) > theta.
 *             After a step, adjacent i, j satisfy x_i' <= 1/(1+a) and x_j' <= 1/(1+gamma^2/a)
 *             for some a > 0 (Def. WRGN), so both >= 1-theta forces gamma <= theta/(1-theta):
 *             under the condition the rounded set {x > 1/2} is independent;
 *   residual: max_i |x_i^{k+1} - x_i^k| <= tol.
 * x0 == NULL selects x0_i = 1/(deg_i + 1).  x0 must be finite, >= 0 and
 * normalizable (Def. 1: (A + I) x0 > 0). */
int gno_run(int n, const int32_t* rp, const int32_t* ci, const double* w, const double* x0,
            int max_iters, double tol, const gno_params* p, int start_iter, double* x_out,
            gno_info* info, double* trace_obj, double* trace_energy, int trace_len) {
  gno_info loc;
  memset(&loc, 0, sizeof loc);
  if (!info) info = &loc;
  memset(info, 0, sizeof *info);
  if (n < 0 || !p || p->check_every < 1 || start_iter < 0 || max_iters < start_iter || !x_out)
    return info->status = GNO_ERR_ARG;
  int st = gno_validate(n, rp, ci, w);
  if (st != GNO_OK) return info->status = st;

  double* v = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* x = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* xn = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) v[i] = sqrt(w[i]);
  for (int i = 0; i < n; ++i) x[i] = x0 ? x0[i] : 1.0 / (double)(rp[i + 1] - rp[i] + 1);

  /* Def. 1: x >= 0 and (A + I) x > 0 */
  for (int i = 0; i < n; ++i) {
    if (!isfinite(x[i]) || x[i] < 0.0) { st = GNO_ERR_NOT_NORMALIZABLE; break; }
  }
  if (st == GNO_OK) {
    for (int i = 0; i < n; ++i) {
      double s = x[i];
      for (int e = rp[i]; e < rp[i + 1]; ++e) s += x[ci[e]];
      if (!(s > 0.0)) { st = GNO_ERR_NOT_NORMALIZABLE; break; }
    }
  }
  if (st != GNO_OK) { free(v); free(x); free(xn); return info->status = st; }

  int stopped = 0, binary_ok = 0, nonbinary = 0;
  long long hits = 0;
  int k = start_iter;
  for (; k < max_iters; ++k) {
    double g = gno_gamma(p, k);
    int t = k - start_iter;
    int chk = is_check(k, p->check_every, max_iters);
    double e_in = (chk || (trace_energy && t < trace_len)) ? gno_energy(n, rp, ci, w, g, x) : 0.0;
    gno_step(n, rp, ci, v, g, x, xn, &hits);
    double rinf = 0.0, rl1 = 0.0;
    nonbinary = 0;
    for (int i = 0; i < n; ++i) {
      double dlt = fabs(xn[i] - x[i]);
      if (dlt > rinf) rinf = dlt;
      rl1 += dlt;
      if (xn[i] > p->theta_bin && xn[i] < 1.0 - p->theta_bin) ++nonbinary;
    }
    if (trace_obj && t < trace_len) trace_obj[t] = gno_objective(n, w, xn);
    if (trace_energy && t < trace_len) trace_energy[t] = e_in;
    double* tmp = x; x = xn; xn = tmp;
    info->resid_inf = rinf;
    info->resid_l1 = rl1;
    info->energy = e_in;
    if (chk) {
      binary_ok = (nonbinary == 0) && (g * (1.0 - p->theta_bin) > p->theta_bin);
      info->binary = (nonbinary == 0);
      if (binary_ok || rinf <= tol) { stopped = 1; ++k; break; }
    }
  }
  info->iters = k - start_iter;
  if (info->iters == 0) {
    nonbinary = 0;
    for (int i = 0; i < n; ++i)
      if (x[i] > p->theta_bin && x[i] < 1.0 - p->theta_bin) ++nonbinary;
    info->binary = (nonbinary == 0);
  }
  for (int i = 0; i < n; ++i) x_out[i] = x[i] < 0.0 ? 0.0 : (x[i] > 1.0 ? 1.0 : x[i]);
  info->objective = gno_objective(n, w, x_out);
  info->safe_div_hits = hits;
  info->converged = stopped;
  if (!stopped) st = GNO_WARN_NOT_CONVERGED;
  else st = binary_ok ? GNO_OK : GNO_WARN_NOT_BINARY;
  free(v); free(x); free(xn);
  return info->status = st;
}

/* Sec. 2 (independent sets) and Sec. 6 ("valid MIS after rounding"): S = {i : x_i > 1/2};
 * S is independent iff no edge has both ends in S; maximal iff every vertex outside S
 * has a neighbour in S.  W(S) = sum_{i in S} w_i in increasing vertex order. */
int gno_extract_is(int n, const int32_t* rp, const int32_t* ci, const double* w,
                   const double* x, uint8_t* mask, int32_t* members, int32_t* count,
                   double* weight) {
  int c = 0;
  double W = 0.0;
  for (int i = 0; i < n; ++i) {
    mask[i] = x[i] > 0.5 ? 1 : 0;
    if (mask[i]) {
      if (members) members[c] = i;
      ++c;
      W += w[i];
    }
  }
  if (count) *count = c;
  if (weight) *weight = W;
  for (int i = 0; i < n; ++i)
    if (mask[i])
      for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (mask[ci[e]]) return GNO_ERR_NOT_INDEPENDENT;
  for (int i = 0; i < n; ++i) {
    if (mask[i]) continue;
    int covered = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (mask[ci[e]]) { covered = 1; break; }
    if (!covered) return GNO_WARN_NOT_MAXIMAL;
  }
  return GNO_OK;
}

/* Thm. 4, eq. (mis-stability): stab(M) = gamma * min_{i not in M} sum_{j in N(i) cap M}
 * sqrt(w_j / w_i).  Returns +inf when every vertex is in M. */
double gno_stability(int n, const int32_t* rp, const int32_t* ci, const double* w,
                     double gamma, const uint8_t* mask) {
  double best = INFINITY;
  for (int i = 0; i < n; ++i) {
    if (mask[i]) continue;
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = ci[e];
      if (mask[j]) s += sqrt(w[j] / w[i]);
    }
    if (s < best) best = s;
  }
  return gamma * best;
}

/* Brute force over every independent set (n <= 31): the maximum weight W* and the
 * maximisers (weights within rel_tol * W* of W*), by include/exclude recursion in
 * vertex order.  Used to bound GN results on tiny graphs (Thm. 4, optimality). */
typedef struct {
  int n;
  const uint32_t* nbr;
  const double* w;
  double rel_tol;
  double best;
  int max_out, n_best;
  uint32_t* out;
} enum_ctx;

static void enum_rec(enum_ctx* c, int i, uint32_t cur, uint32_t blocked, double wsum) {
  if (i == c->n) {
    double tol = c->rel_tol * (c->best > 0 ? c->best : 1.0);
    if (wsum > c->best + tol) {
      c->best = wsum;
      c->n_best = 0;
    }
    if (fabs(wsum - c->best) <= c->rel_tol * (c->best > 0 ? c->best : 1.0)) {
      if (c->n_best < c->max_out && c->out) c->out[c->n_best] = cur;
      c->n_best++;
    }
    return;
  }
  enum_rec(c, i + 1, cur, blocked, wsum);
  if (!(blocked & (1u << i)))
    enum_rec(c, i + 1, cur | (1u << i), blocked | c->nbr[i] | (1u << i), wsum + c->w[i]);
}

int gno_mwis_enumerate(int n, const int32_t* rp, const int32_t* ci, const double* w,
                       double rel_tol, int max_out, uint32_t* masks_out, int* n_best,
                       double* best_weight) {
  if (n < 0 || n > 31) return GNO_ERR_ARG;
  uint32_t nbr[32];
  for (int i = 0; i < n; ++i) {
    nbr[i] = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) nbr[i] |= 1u << ci[e];
  }
  enum_ctx c = {n, nbr, w, rel_tol, -INFINITY, max_out, 0, masks_out};
  /* two passes: the first finds W*, the second collects every maximiser */
  enum_rec(&c, 0, 0u, 0u, 0.0);
  double best = c.best;
  c.n_best = 0;
  c.best = best;
  enum_rec(&c, 0, 0u, 0u, 0.0);
  if (n_best) *n_best = c.n_best;
  if (best_weight) *best_weight = best;
  return GNO_OK;
}

/* Textbook Hungarian method (Kuhn; shortest augmenting paths with row and column
 * potentials) for the k x k assignment problem, minimising sum_i cost[i*k + assign[i]].
 * The paper names it as the exact solver of the assignment problem (Sec. 1).  O(k^3). */
double gno_hungarian(int k, const double* cost, int32_t* assign) {
  /* 1-based arrays: u (rows), vv (columns), match[col] = row, prev[col] = previous column */
  double* u = (double*)calloc((size_t)k + 1, sizeof(double));
  double* vv = (double*)calloc((size_t)k + 1, sizeof(double));
  double* dist = (double*)malloc(sizeof(double) * ((size_t)k + 1));
  int* match = (int*)calloc((size_t)k + 1, sizeof(int));
  int* prev = (int*)calloc((size_t)k + 1, sizeof(int));
  char* used = (char*)malloc((size_t)k + 1);
  for (int r = 1; r <= k; ++r) {
    match[0] = r;           /* column 0 is a virtual start holding the new row */
    int c0 = 0;
    for (int c = 0; c <= k; ++c) { dist[c] = INFINITY; used[c] = 0; }
    do {
      used[c0] = 1;
      int r0 = match[c0], c1 = 0;
      double delta = INFINITY;
      for (int c = 1; c <= k; ++c) {
        if (used[c]) continue;
        double red = cost[(size_t)(r0 - 1) * k + (c - 1)] - u[r0] - vv[c];
        if (red < dist[c]) { dist[c] = red; prev[c] = c0; }
        if (dist[c] < delta) { delta = dist[c]; c1 = c; }
      }
      for (int c = 0; c <= k; ++c) {
        if (used[c]) { u[match[c]] += delta; vv[c] -= delta; }
        else dist[c] -= delta;
      }
      c0 = c1;
    } while (match[c0] != 0);
    do {                    /* flip the augmenting path back to the virtual column */
      int c1 = prev[c0];
      match[c0] = match[c1];
      c0 = c1;
    } while (c0 != 0);
  }
  double total = 0.0;
  for (int c = 1; c <= k; ++c) {
    assign[match[c] - 1] = c - 1;
  }
  for (int r = 0; r < k; ++r) total += cost[(size_t)r * k + assign[r]];
  free(u); free(vv); free(dist); free(match); free(prev); free(used);
  return total;
}
