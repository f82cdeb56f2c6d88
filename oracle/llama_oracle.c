/*
 * llama_oracle.c -- CPU oracle of Llama's per-invocation scheduling step
 * (arXiv 2102.01887: slack allotment, Section 4.1 / Algorithm 1; cost-based
 * configuration selection, Section 4.2 / Eq. 1).
 *
 * TEST INFRASTRUCTURE.  This file exists to check the CUDA path, never to
 * serve it: only the tests, the package smoke check and the benchmark's CPU
 * baseline may load it.  It is plain, single-threaded, slow on purpose, and
 * shares no code, header, table or constant with the CUDA library.
 *
 * Integer readings of the paper (all times int64 microseconds, costs int64
 * nano-dollars; intermediate products in 128-bit so nothing can overflow):
 *   - elapsed time t of an invocation = now - start of its pipeline instance;
 *   - remaining time  R(lambda) = target - t - queueingTime(lambda)  (Alg. 1);
 *   - remaining path latency of op on a path = sum of reference latencies of
 *     op and every operation after it on that path (Section 4.1: "starting
 *     at op", so op itself is included);
 *   - per-path slack = floor(ref(op) * R / RemainingPathLatency), the minimum
 *     over all source-to-sink paths through op is the slack (Alg. 1);
 *     when R <= 0 the target has already passed and the slack is 0;
 *   - a configuration x is feasible when L(x) < slack(op, lambda(x)), the
 *     strict test of Eq. 1's first case;
 *   - cost-first mode: among feasible configurations the lowest cost wins;
 *     if none is feasible the lowest latency wins; ties go to the lowest
 *     configuration index;
 *   - alpha mode: Eq. 1 in integers, obj = C/B when feasible, otherwise
 *     C/B + floor(alpha_num * L * R(x) / (alpha_den * B(x) * R_total)),
 *     saturating at INT64_MAX; argmin over (obj, index).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ETOOBIG (-6)

#define OR_MODE_COST_FIRST 0
#define OR_MODE_ALPHA 1

#define OR_FLAG_FEASIBLE 1
#define OR_FLAG_INVALID 2

#define OR_SLACK_BY_CRITICAL_PATH 0
#define OR_SLACK_BY_PATHS 1

typedef struct {
    int32_t n_dags, n_ops, n_hw, mode;
    const int32_t *dag_op_off; /* [n_dags+1] */
    const int32_t *row_ptr;    /* [n_ops+1]  successors, global op ids */
    const int32_t *col;        /* [n_edges] */
    const int64_t *slo_us;     /* [n_dags]   pipeline latency target */
    const int64_t *cfg_off;    /* [n_ops+1] */
    const int32_t *hw_off;     /* [n_ops*(n_hw+1)], op-local segment starts */
    const int32_t *lat_us;     /* [n_cfg] L(x) */
    const int64_t *cost_nd;    /* [n_cfg] C(x)/B(x) */
    const int32_t *ref_cfg;    /* [n_ops] op-local reference configuration */
    const int32_t *batch;      /* [n_cfg] B(x), alpha mode only */
    const int32_t *res;        /* [n_cfg] R(x), alpha mode only */
    const int32_t *res_total;  /* [n_hw]  R_total(lambda), alpha mode only */
    const int64_t *q_us;       /* [n_hw]  queueingTime(lambda) */
    int64_t alpha_num, alpha_den;
} or_problem;

typedef struct {
    int32_t cfg;   /* op-local index of the chosen configuration, -1 if invalid */
    int32_t lat;   /* L(cfg) */
    int64_t cost;  /* C(cfg)/B(cfg) */
    int32_t slack; /* slack(op, lambda(cfg)) */
    int32_t flags; /* OR_FLAG_* */
} or_decision;

/* Reference latency of operation v: the latency of its reference
 * configuration (Section 3.2, smallest CPU configuration). */
static int64_t ref_latency(const or_problem *p, int32_t v) {
    return (int64_t)p->lat_us[p->cfg_off[v] + p->ref_cfg[v]];
}

/* Kahn's algorithm over the successor CSR; fails on a cycle. */
int or_topo_order(int32_t n_ops, const int32_t *row_ptr, const int32_t *col, int32_t *order) {
    int32_t *indeg = calloc((size_t)n_ops + 1, sizeof(int32_t));
    if (!indeg) return OR_ENOMEM;
    for (int32_t v = 0; v < n_ops; v++)
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) indeg[col[e]]++;
    int32_t head = 0, tail = 0;
    for (int32_t v = 0; v < n_ops; v++)
        if (indeg[v] == 0) order[tail++] = v;
    while (head < tail) {
        int32_t v = order[head++];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++)
            if (--indeg[col[e]] == 0) order[tail++] = col[e];
    }
    free(indeg);
    return tail == n_ops ? OR_OK : OR_EINVAL;
}

/* Longest remaining path latency from every operation to a sink, op
 * included: cp[v] = ref[v] + max over successors w of cp[w] (0 at a sink).
 * For R >= 0 the minimum of Algorithm 1 over paths is attained on the path
 * with the largest RemainingPathLatency, which is cp[v]. */
int or_critical_path(int32_t n_ops, const int32_t *row_ptr, const int32_t *col,
                     const int64_t *ref, int64_t *cp) {
    int32_t *order = malloc(((size_t)n_ops + 1) * sizeof(int32_t));
    if (!order) return OR_ENOMEM;
    int rc = or_topo_order(n_ops, row_ptr, col, order);
    if (rc == OR_OK) {
        for (int32_t i = n_ops - 1; i >= 0; i--) {
            int32_t v = order[i];
            int64_t best = 0;
            for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++)
                if (cp[col[e]] > best) best = cp[col[e]];
            cp[v] = ref[v] + best;
        }
    }
    free(order);
    return rc;
}

/* Per-path slack of Algorithm 1 in integers: floor(ref * R / pLat), with the
 * passed-target case (R <= 0) giving 0. */
static int64_t path_slack(int64_t ref, int64_t rem_path, int64_t R) {
    if (R <= 0) return 0;
    __int128 num = (__int128)ref * (__int128)R;
    return (int64_t)(num / rem_path);
}

int64_t or_slack_from_cp(int64_t ref, int64_t cp, int64_t R) { return path_slack(ref, cp, R); }

/* Algorithm 1 taken literally: enumerate every source-to-sink path of the
 * DAG whose operations are [first, last) (the Pipeline-Decomposer's
 * depth-first search, Section 3.2), keep the paths that contain op, and
 * return the minimum per-path slack.  Fails with OR_ETOOBIG after max_paths
 * paths. */
int or_slack_paths(int32_t first, int32_t last, const int32_t *row_ptr, const int32_t *col,
                   const int64_t *ref, int32_t op, int64_t R, int64_t max_paths,
                   int64_t *slack, int64_t *n_paths) {
    int32_t n = last - first;
    int rc = OR_OK;
    int32_t *indeg = calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *path = malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *next_edge = malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!indeg || !path || !next_edge) { rc = OR_ENOMEM; goto done; }
    for (int32_t v = first; v < last; v++)
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) indeg[col[e] - first]++;
    int64_t best = INT64_MAX, count = 0;
    for (int32_t s = first; s < last; s++) {
        if (indeg[s - first] != 0) continue;          /* not an input operation */
        int32_t depth = 0;
        path[0] = s;
        next_edge[0] = row_ptr[s];
        while (depth >= 0) {
            int32_t v = path[depth];
            if (row_ptr[v] == row_ptr[v + 1]) {       /* v is an output operation: path complete */
                if (++count > max_paths) { rc = OR_ETOOBIG; goto done; }
                int32_t pos = -1;
                for (int32_t k = 0; k <= depth; k++)
                    if (path[k] == op) pos = k;
                if (pos >= 0) {
                    int64_t rem = 0;
                    for (int32_t k = pos; k <= depth; k++) rem += ref[path[k]];
                    int64_t ps = path_slack(ref[op], rem, R);
                    if (ps < best) best = ps;
                }
                depth--;
                continue;
            }
            if (next_edge[depth] < row_ptr[v + 1]) {
                int32_t w = col[next_edge[depth]++];
                depth++;
                path[depth] = w;
                next_edge[depth] = row_ptr[w];
            } else {
                depth--;
            }
        }
    }
    if (best == INT64_MAX) rc = OR_EINVAL;           /* op lies on no path */
    *slack = best;
    *n_paths = count;
done:
    free(indeg);
    free(path);
    free(next_edge);
    return rc;
}

/* Hardware backend lambda(x) of op-local configuration x of operation v. */
static int32_t backend_of(const or_problem *p, int32_t v, int32_t x) {
    const int32_t *off = p->hw_off + (int64_t)v * (p->n_hw + 1);
    for (int32_t h = 0; h < p->n_hw; h++)
        if (x >= off[h] && x < off[h + 1]) return h;
    return -1;
}

/* Eq. 1's second case in integers, saturating at INT64_MAX. */
static int64_t alpha_objective_infeasible(const or_problem *p, int64_t g, int32_t h) {
    unsigned __int128 num = (unsigned __int128)p->alpha_num * (unsigned __int128)p->lat_us[g]
                            * (unsigned __int128)p->res[g];
    unsigned __int128 den = (unsigned __int128)p->alpha_den * (unsigned __int128)p->batch[g]
                            * (unsigned __int128)p->res_total[h];
    unsigned __int128 obj = (unsigned __int128)p->cost_nd[g] + num / den;
    return obj > (unsigned __int128)INT64_MAX ? INT64_MAX : (int64_t)obj;
}

/* Score every configuration of operation v against the slack of its backend
 * and keep the best one by plain comparisons (Section 4.2: Eq. 1 is applied
 * to all configurations x of op, each with slack(op, lambda(x))). */
int or_select(const or_problem *p, int32_t v, const int64_t *slack_hw, or_decision *out) {
    int64_t first = p->cfg_off[v];
    int32_t n = (int32_t)(p->cfg_off[v + 1] - first);
    int32_t best = -1, best_feasible = 0;
    int64_t best_obj = 0;
    for (int32_t x = 0; x < n; x++) {
        int64_t g = first + x;
        int32_t h = backend_of(p, v, x);
        if (h < 0) return OR_EINVAL;
        int feasible = (int64_t)p->lat_us[g] < slack_hw[h];
        int take = 0;
        if (p->mode == OR_MODE_ALPHA) {
            int64_t obj = feasible ? p->cost_nd[g] : alpha_objective_infeasible(p, g, h);
            if (best < 0 || obj < best_obj) { take = 1; best_obj = obj; }
        } else {
            if (best < 0) take = 1;
            else if (feasible && !best_feasible) take = 1;
            else if (feasible && best_feasible) take = p->cost_nd[g] < p->cost_nd[first + best];
            else if (!feasible && !best_feasible) take = p->lat_us[g] < p->lat_us[first + best];
        }
        if (take) { best = x; best_feasible = feasible; }
    }
    if (best < 0) return OR_EINVAL;
    int64_t g = first + best;
    out->cfg = best;
    out->lat = p->lat_us[g];
    out->cost = p->cost_nd[g];
    out->slack = (int32_t)slack_hw[backend_of(p, v, best)];
    out->flags = best_feasible ? OR_FLAG_FEASIBLE : 0;
    return OR_OK;
}

static int invocation_valid(const or_problem *p, int32_t d, int32_t op_local, int64_t start, int64_t now) {
    if (d < 0 || d >= p->n_dags) return 0;
    if (op_local < 0 || op_local >= p->dag_op_off[d + 1] - p->dag_op_off[d]) return 0;
    if (start < 0 || start > now) return 0;
    return 1;
}

/* Slack of every invocation for every backend, int64[n_inv * n_hw]; invalid
 * invocations get -1. */
int or_slacks(const or_problem *p, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
              const int64_t *start, int64_t now, int32_t method, int64_t *slack_out) {
    int64_t *ref = malloc(((size_t)p->n_ops + 1) * sizeof(int64_t));
    int64_t *cp = malloc(((size_t)p->n_ops + 1) * sizeof(int64_t));
    int rc = (ref && cp) ? OR_OK : OR_ENOMEM;
    if (rc == OR_OK) {
        for (int32_t v = 0; v < p->n_ops; v++) ref[v] = ref_latency(p, v);
        rc = or_critical_path(p->n_ops, p->row_ptr, p->col, ref, cp);
    }
    for (int64_t i = 0; rc == OR_OK && i < n_inv; i++) {
        if (!invocation_valid(p, dag[i], op_local[i], start[i], now)) {
            for (int32_t h = 0; h < p->n_hw; h++) slack_out[i * p->n_hw + h] = -1;
            continue;
        }
        int32_t v = p->dag_op_off[dag[i]] + op_local[i];
        int64_t t = now - start[i];
        for (int32_t h = 0; h < p->n_hw; h++) {
            int64_t R = p->slo_us[dag[i]] - t - p->q_us[h];
            int64_t s;
            if (method == OR_SLACK_BY_PATHS) {
                int64_t np_;
                rc = or_slack_paths(p->dag_op_off[dag[i]], p->dag_op_off[dag[i] + 1], p->row_ptr,
                                    p->col, ref, v, R, 1000000, &s, &np_);
                if (rc != OR_OK) break;
            } else {
                s = or_slack_from_cp(ref[v], cp[v], R);
            }
            slack_out[i * p->n_hw + h] = s;
        }
    }
    free(ref);
    free(cp);
    return rc;
}

/* The whole scheduling step for a batch of pending invocations: slack per
 * backend (Algorithm 1), then configuration selection (Eq. 1).  Invalid
 * invocations get cfg = -1 and OR_FLAG_INVALID; the call then returns
 * OR_EINVAL after filling every valid one. */
int or_schedule(const or_problem *p, int64_t n_inv, const int32_t *dag, const int32_t *op_local,
                const int64_t *start, int64_t now, int32_t method, or_decision *out) {
    int64_t *slack = malloc(((size_t)n_inv * p->n_hw + 1) * sizeof(int64_t));
    if (!slack) return OR_ENOMEM;
    int rc = or_slacks(p, n_inv, dag, op_local, start, now, method, slack);
    int any_invalid = 0;
    for (int64_t i = 0; rc == OR_OK && i < n_inv; i++) {
        if (!invocation_valid(p, dag[i], op_local[i], start[i], now)) {
            out[i].cfg = -1;
            out[i].lat = 0;
            out[i].cost = 0;
            out[i].slack = 0;
            out[i].flags = OR_FLAG_INVALID;
            any_invalid = 1;
            continue;
        }
        rc = or_select(p, p->dag_op_off[dag[i]] + op_local[i], slack + i * p->n_hw, &out[i]);
    }
    free(slack);
    if (rc == OR_OK && any_invalid) rc = OR_EINVAL;
    return rc;
}
