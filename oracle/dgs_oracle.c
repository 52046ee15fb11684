/*
 * dgs_oracle.c -- plain CPU oracle for Deep Greedy Switching (single-threaded
 * by default; see oracle_set_evaluation).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the CUDA library.  Written for
 * readability against the paper, not for speed: no blocking, no fusion, no
 * incremental tricks.  Every function names the part of the paper it follows.
 *
 * Storage: a[i*n + j] = benefit of agent i doing job j (int32, |a| < 2^29).
 * sigma[j] = agent holding job j, tau[i] = job held by agent i (Section 3.3).
 */
#include "dgs_oracle.h"

#include <stdlib.h>
#include <string.h>

#define ORACLE_ERR_INTERNAL 99
#define A(i, j) ((int64_t)a[(int64_t)(i) * n + (j)])

/* Section 3: f(sigma) = sum over agents of the benefit of their job. */
int64_t oracle_objective(const int32_t* a, int32_t n, const int32_t* tau)
{
    int64_t f = 0;
    for (int32_t i = 0; i < n; ++i) f += A(i, tau[i]);
    return f;
}

int oracle_range_ok(const int32_t* a, int32_t n)
{
    const int64_t lim = (int64_t)1 << 29;
    for (int64_t e = 0; e < (int64_t)n * n; ++e)
        if (a[e] >= lim || a[e] <= -lim) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Section 3.1, reading R1: global greedy.  Visit all (i, j) pairs by
 * decreasing benefit (ties: lower agent first, then lower job) and take a
 * pair whenever both its agent and its job are still free.  The order is
 * encoded in one unsigned 64-bit sort key per pair:
 *   bits 34..63: (2^30 - 1) - (a + 2^29)   (larger benefit -> smaller key)
 *   bits 17..33: agent i,  bits 0..16: job j          (n <= 2^17)       */
static int cmp_u64(const void* x, const void* y)
{
    uint64_t u = *(const uint64_t*)x, v = *(const uint64_t*)y;
    return (u > v) - (u < v);
}

void oracle_greedy_init(const int32_t* a, int32_t n, int32_t* tau_out)
{
    int64_t m = (int64_t)n * n;
    uint64_t* keys = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
    uint8_t* agent_used = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* job_used = (uint8_t*)calloc((size_t)n, 1);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) {
            uint64_t rank = (uint64_t)(((int64_t)1 << 30) - 1 - (A(i, j) + ((int64_t)1 << 29)));
            keys[(int64_t)i * n + j] = (rank << 34) | ((uint64_t)i << 17) | (uint64_t)j;
        }
    qsort(keys, (size_t)m, sizeof(uint64_t), cmp_u64);
    int32_t taken = 0;
    for (int64_t e = 0; e < m && taken < n; ++e) {
        int32_t i = (int32_t)((keys[e] >> 17) & 0x1FFFF);
        int32_t j = (int32_t)(keys[e] & 0x1FFFF);
        if (!agent_used[i] && !job_used[j]) {
            agent_used[i] = 1;
            job_used[j] = 1;
            tau_out[i] = j;
            ++taken;
        }
    }
    free(keys);
    free(agent_used);
    free(job_used);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 (ADE) for agent i.  j = tau(i).  For every other job j'
 * (ascending, reading R2) with holder i' = sigma(j'), the candidate
 * assignment gives j' to i and j to i'; it is kept when its objective is
 * strictly larger than the best kept so far (initially sigma itself).  The
 * objective difference of that candidate against sigma is the four-term
 * expression below (only agents i and i' change jobs). */
void oracle_ade(const int32_t* a, int32_t n, const int32_t* sigma,
                const int32_t* tau, int32_t i, int32_t* gain, int32_t* job)
{
    int32_t j = tau[i];
    int64_t best = 0;
    int32_t best_job = -1;
    for (int32_t jp = 0; jp < n; ++jp) {
        if (jp == j) continue;
        int32_t ip = sigma[jp];
        int64_t diff = A(i, jp) + A(ip, j) - A(i, j) - A(ip, jp);
        if (diff > best) {
            best = diff;
            best_job = jp;
        }
    }
    *gain = (int32_t)best;
    *job = best_job;
}

/* JDE for job j (Section 3.2): job j, held by i = sigma(j), tries every
 * other agent i' (ascending, reading R2); the candidate gives j to i' and
 * i's partner job j' = tau(i') to i. */
void oracle_jde(const int32_t* a, int32_t n, const int32_t* sigma,
                const int32_t* tau, int32_t j, int32_t* gain, int32_t* agent)
{
    int32_t i = sigma[j];
    int64_t best = 0;
    int32_t best_agent = -1;
    for (int32_t ip = 0; ip < n; ++ip) {
        if (ip == i) continue;
        int32_t jp = tau[ip];
        int64_t diff = A(ip, j) + A(i, jp) - A(i, j) - A(ip, jp);
        if (diff > best) {
            best = diff;
            best_agent = ip;
        }
    }
    *gain = (int32_t)best;
    *agent = best_agent;
}

void oracle_evaluate_all(const int32_t* a, int32_t n, const int32_t* tau,
                         int32_t* agent_gain, int32_t* agent_job,
                         int32_t* job_gain, int32_t* job_agent)
{
    int32_t* sigma = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int32_t i = 0; i < n; ++i) sigma[tau[i]] = i;
    for (int32_t i = 0; i < n; ++i) oracle_ade(a, n, sigma, tau, i, &agent_gain[i], &agent_job[i]);
    for (int32_t j = 0; j < n; ++j) oracle_jde(a, n, sigma, tau, j, &job_gain[j], &job_agent[j]);
    free(sigma);
}

/* ------------------------------------------------------------------------ */
/* How the slot evaluations of Algorithm 3 are carried out.  Algorithm 3
 * evaluates every agent and every job "in parallel": each ADE/JDE reads the
 * current assignment and writes only its own slot, so running them on
 * several host threads changes no result.  With use_transpose the column
 * entries a[i'][j] of the four-term difference are read from a plain
 * transposed copy at[j][i'] (the same integers, contiguous in memory).
 * Defaults: one thread, no copy -- the literal loops above.  Only the
 * script that writes stored full-size results changes them; the tests check
 * that every setting gives the same solve. */
static int32_t g_eval_threads = 1;
static int32_t g_eval_transpose = 0;

void oracle_set_evaluation(int32_t threads, int32_t use_transpose)
{
    g_eval_threads = threads > 1 ? threads : 1;
    g_eval_transpose = use_transpose ? 1 : 0;
}

#define AT(j, i) ((int64_t)at[(int64_t)(j) * n + (i)])

/* oracle_ade with a[i'][j] read as at[j][i']. */
static void ade_transposed(const int32_t* a, const int32_t* at, int32_t n, const int32_t* sigma,
                           const int32_t* tau, int32_t i, int32_t* gain, int32_t* job)
{
    int32_t j = tau[i];
    int64_t best = 0;
    int32_t best_job = -1;
    for (int32_t jp = 0; jp < n; ++jp) {
        if (jp == j) continue;
        int32_t ip = sigma[jp];
        int64_t diff = A(i, jp) + AT(j, ip) - A(i, j) - A(ip, jp);
        if (diff > best) {
            best = diff;
            best_job = jp;
        }
    }
    *gain = (int32_t)best;
    *job = best_job;
}

/* oracle_jde with a[i'][j] read as at[j][i'] and a[i'][j'] as at[j'][i']. */
static void jde_transposed(const int32_t* a, const int32_t* at, int32_t n, const int32_t* sigma,
                           const int32_t* tau, int32_t j, int32_t* gain, int32_t* agent)
{
    int32_t i = sigma[j];
    int64_t best = 0;
    int32_t best_agent = -1;
    for (int32_t ip = 0; ip < n; ++ip) {
        if (ip == i) continue;
        int32_t jp = tau[ip];
        int64_t diff = AT(j, ip) + A(i, jp) - A(i, j) - AT(jp, ip);
        if (diff > best) {
            best = diff;
            best_agent = ip;
        }
    }
    *gain = (int32_t)best;
    *agent = best_agent;
}

/* ADE of every agent i with pick_a == NULL or pick_a[i] == 0, and JDE of
 * every job j with pick_j == NULL or pick_j[j] == 0; returns how many ran. */
static int64_t evaluate_slots(const int32_t* a, const int32_t* at, int32_t n, const int32_t* sigma,
                              const int32_t* tau, const uint8_t* pick_a, const uint8_t* pick_j,
                              int32_t* ag_gain, int32_t* ag_job, int32_t* jb_gain, int32_t* jb_agent)
{
    int64_t count = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_eval_threads) if (g_eval_threads > 1)
    for (int32_t i = 0; i < n; ++i) {
        if (pick_a && pick_a[i]) continue;
        if (at) ade_transposed(a, at, n, sigma, tau, i, &ag_gain[i], &ag_job[i]);
        else oracle_ade(a, n, sigma, tau, i, &ag_gain[i], &ag_job[i]);
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_eval_threads) if (g_eval_threads > 1)
    for (int32_t j = 0; j < n; ++j) {
        if (pick_j && pick_j[j]) continue;
        if (at) jde_transposed(a, at, n, sigma, tau, j, &jb_gain[j], &jb_agent[j]);
        else oracle_jde(a, n, sigma, tau, j, &jb_gain[j], &jb_agent[j]);
    }
    for (int32_t t = 0; t < n; ++t) count += (!pick_a || !pick_a[t]) + (!pick_j || !pick_j[t]);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 4 (CC), reading R3.  CR collects claimed agents.  Agent slots
 * are visited first (ascending i), then job slots (ascending j); a slot
 * with a candidate claims the two agents its exchange touches -- for agent
 * slot i: i and i' = sigma(j_i); for job slot j: sigma(j) and i_j -- unless
 * one of them is already claimed, in which case the slot goes into C.
 * Partners are looked up in the current sigma. */
void oracle_check_conflicts(int32_t n, const int32_t* sigma,
                            const int32_t* agent_gain, const int32_t* agent_job,
                            const int32_t* job_gain, const int32_t* job_agent,
                            uint8_t* in_ca, uint8_t* in_cj)
{
    uint8_t* cr = (uint8_t*)calloc((size_t)n, 1);
    for (int32_t i = 0; i < n; ++i) {
        in_ca[i] = 0;
        if (agent_gain[i] <= 0) continue; /* NA_i = 0 */
        int32_t ip = sigma[agent_job[i]];
        if (cr[i] || cr[ip]) {
            in_ca[i] = 1;
        } else {
            cr[i] = 1;
            cr[ip] = 1;
        }
    }
    for (int32_t j = 0; j < n; ++j) {
        in_cj[j] = 0;
        if (job_gain[j] <= 0) continue; /* NJ_j = 0 */
        int32_t owner = sigma[j];
        int32_t partner = job_agent[j];
        if (cr[owner] || cr[partner]) {
            in_cj[j] = 1;
        } else {
            cr[owner] = 1;
            cr[partner] = 1;
        }
    }
    free(cr);
}

/* Literal Algorithm 4: C is a set of AGENTS; a conflicted job slot adds its
 * owner sigma(j).  Kept only to demonstrate that this reading never lets the
 * switching loop finish (see the tests). */
static void cc_literal_agents(int32_t n, const int32_t* sigma,
                              const int32_t* agent_gain, const int32_t* agent_job,
                              const int32_t* job_gain, const int32_t* job_agent,
                              uint8_t* in_c_agent)
{
    uint8_t* cr = (uint8_t*)calloc((size_t)n, 1);
    memset(in_c_agent, 0, (size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        if (agent_gain[i] <= 0) continue;
        int32_t ip = sigma[agent_job[i]];
        if (cr[i] || cr[ip]) in_c_agent[i] = 1;
        else { cr[i] = 1; cr[ip] = 1; }
    }
    for (int32_t j = 0; j < n; ++j) {
        if (job_gain[j] <= 0) continue;
        int32_t owner = sigma[j];
        if (cr[owner] || cr[job_agent[j]]) in_c_agent[owner] = 1;
        else { cr[owner] = 1; cr[job_agent[j]] = 1; }
    }
    free(cr);
}

/* Objective change of exchanging the jobs of agents u and v under tau. */
static int64_t exchange_gain(const int32_t* a, int32_t n, const int32_t* tau,
                             int32_t u, int32_t v)
{
    return A(u, tau[v]) + A(v, tau[u]) - A(u, tau[u]) - A(v, tau[v]);
}

static void do_exchange(int32_t* sigma, int32_t* tau, int32_t u, int32_t v)
{
    int32_t ju = tau[u], jv = tau[v];
    tau[u] = jv;
    tau[v] = ju;
    sigma[jv] = u;
    sigma[ju] = v;
}

/* ------------------------------------------------------------------------ */
/* Random start (Section 3.1): splitmix64 (Steele, Lea, Flood 2014) and the
 * Fisher-Yates shuffle in Durstenfeld's form. */
uint64_t oracle_splitmix64_next(uint64_t* state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void oracle_random_permutation(int32_t n, uint64_t seed, int32_t* tau_out)
{
    uint64_t state = seed;
    for (int32_t i = 0; i < n; ++i) tau_out[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)(oracle_splitmix64_next(&state) % (uint64_t)(i + 1));
        int32_t t = tau_out[i];
        tau_out[i] = tau_out[j];
        tau_out[j] = t;
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 3 (parallel DGS). */
int oracle_dgs_parallel(const int32_t* a, int32_t n, int32_t init_mode,
                        const int32_t* init_tau, uint64_t seed, int32_t max_sweeps,
                        int32_t cc_rule, int32_t reeval_rule, int32_t* tau_out, int64_t* f_out,
                        oracle_stats* stats, int32_t trace_cap,
                        int32_t* trace_accepted, int32_t* trace_applied,
                        int64_t* trace_objective)
{
    if (n <= 0 || a == NULL || tau_out == NULL || f_out == NULL) return ORACLE_ERR_INVALID;
    if (n > (1 << 17)) return ORACLE_ERR_INVALID;
    if (!oracle_range_ok(a, n)) return ORACLE_ERR_RANGE;

    size_t nb = (size_t)n * sizeof(int32_t);
    int32_t* sigma = (int32_t*)malloc(nb);
    int32_t* tau = (int32_t*)malloc(nb);
    int32_t* tau0 = (int32_t*)malloc(nb);
    int32_t* ag_gain = (int32_t*)malloc(nb);
    int32_t* ag_job = (int32_t*)malloc(nb);
    int32_t* jb_gain = (int32_t*)malloc(nb);
    int32_t* jb_agent = (int32_t*)malloc(nb);
    uint8_t* in_ca = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* in_cj = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* in_c_agent = (uint8_t*)calloc((size_t)n, 1);
    int32_t* at = NULL; /* transposed copy, only with oracle_set_evaluation(.., 1) */
    if (g_eval_transpose) {
        at = (int32_t*)malloc((size_t)n * n * sizeof(int32_t));
        for (int32_t i = 0; i < n; ++i)
            for (int32_t j = 0; j < n; ++j) at[(int64_t)j * n + i] = a[(int64_t)i * n + j];
    }
    oracle_stats st = {0, 0, 0, 0};
    int status = ORACLE_OK;

    /* Section 3.1: initial solution. */
    if (init_mode == ORACLE_INIT_GREEDY) {
        oracle_greedy_init(a, n, tau);
    } else if (init_mode == ORACLE_INIT_IDENTITY) {
        for (int32_t i = 0; i < n; ++i) tau[i] = i;
    } else if (init_mode == ORACLE_INIT_RANDOM) {
        oracle_random_permutation(n, seed, tau);
    } else if (init_mode == ORACLE_INIT_USER && init_tau != NULL) {
        memset(in_ca, 0, (size_t)n);
        for (int32_t i = 0; i < n; ++i) {
            if (init_tau[i] < 0 || init_tau[i] >= n || in_ca[init_tau[i]]) {
                status = ORACLE_ERR_INVALID;
                goto out;
            }
            in_ca[init_tau[i]] = 1;
            tau[i] = init_tau[i];
        }
        memset(in_ca, 0, (size_t)n);
    } else {
        status = ORACLE_ERR_INVALID;
        goto out;
    }
    for (int32_t i = 0; i < n; ++i) sigma[tau[i]] = i;
    int64_t f = oracle_objective(a, n, tau);

    for (;;) { /* outer repeat ... until f(sigma_start) = f(sigma') (R5) */
        st.passes++;
        int64_t f_start = f;
        memset(in_ca, 0, (size_t)n);
        memset(in_cj, 0, (size_t)n);
        memset(in_c_agent, 0, (size_t)n);

        /* Difference evaluation phase: every agent and every job. */
        st.evaluations += evaluate_slots(a, at, n, sigma, tau, NULL, NULL, ag_gain, ag_job, jb_gain, jb_agent);

        for (;;) { /* switching phase: while some delta > 0 */
            int any = 0;
            for (int32_t t = 0; t < n && !any; ++t) any = ag_gain[t] > 0 || jb_gain[t] > 0;
            if (!any) break;
            if (max_sweeps > 0 && st.sweeps >= max_sweeps) {
                status = ORACLE_TIMEOUT;
                goto finish;
            }

            /* CC, then delta_t = candidate gain of every slot not in C. */
            if (cc_rule == ORACLE_CC_SLOTS) {
                oracle_check_conflicts(n, sigma, ag_gain, ag_job, jb_gain, jb_agent, in_ca, in_cj);
            } else {
                cc_literal_agents(n, sigma, ag_gain, ag_job, jb_gain, jb_agent, in_c_agent);
                for (int32_t i = 0; i < n; ++i) in_ca[i] = in_c_agent[i];
                for (int32_t j = 0; j < n; ++j) in_cj[j] = in_c_agent[sigma[j]];
            }

            /* Parallel switch: every slot with delta_t > 0 performs its
             * exchange if that raises f under the current sigma.  The
             * accepted slots touch disjoint agents, so applying them in slot
             * order equals applying them all against the sigma of the CC;
             * the snapshot comparison checks exactly that. */
            memcpy(tau0, tau, nb);
            int32_t accepted = 0, applied = 0;
            for (int32_t t = 0; t < 2 * n; ++t) {
                int32_t u, v;
                if (t < n) {
                    if (in_ca[t] || ag_gain[t] <= 0) continue;
                    u = t;
                    v = sigma[ag_job[t]];
                } else {
                    int32_t j = t - n;
                    if (in_cj[j] || jb_gain[j] <= 0) continue;
                    u = jb_agent[j];
                    v = sigma[j];
                }
                accepted++;
                int64_t g = exchange_gain(a, n, tau, u, v);
                if (g != exchange_gain(a, n, tau0, u, v)) {
                    status = ORACLE_ERR_INTERNAL;
                    goto finish;
                }
                if (g > 0) {
                    do_exchange(sigma, tau, u, v);
                    f += g;
                    applied++;
                }
            }
            st.swaps_applied += applied;

            /* Re-evaluation of the agents and jobs not in C (reading R4), or
             * of every agent and job (ORACLE_REEVAL_ALL). */
            const int all = reeval_rule == ORACLE_REEVAL_ALL;
            st.evaluations += evaluate_slots(a, at, n, sigma, tau, all ? NULL : in_ca, all ? NULL : in_cj,
                                             ag_gain, ag_job, jb_gain, jb_agent);

            if (st.sweeps < trace_cap) {
                if (trace_accepted) trace_accepted[st.sweeps] = accepted;
                if (trace_applied) trace_applied[st.sweeps] = applied;
                if (trace_objective) trace_objective[st.sweeps] = f;
            }
            st.sweeps++;
        }
        if (f == f_start) break;
    }

finish:
    memcpy(tau_out, tau, nb);
    *f_out = oracle_objective(a, n, tau);
    if (status == ORACLE_OK && *f_out != f) status = ORACLE_ERR_INTERNAL;
out:
    if (stats) *stats = st;
    free(sigma); free(tau); free(tau0);
    free(ag_gain); free(ag_job); free(jb_gain); free(jb_agent);
    free(in_ca); free(in_cj); free(in_c_agent); free(at);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (sequential DGS). */
int oracle_dgs_sequential(const int32_t* a, int32_t n, int32_t init_mode,
                          const int32_t* init_tau, uint64_t seed, int32_t max_iters,
                          int32_t* tau_out, int64_t* f_out, oracle_stats* stats,
                          int32_t trace_cap, int32_t* trace_applied, int64_t* trace_objective,
                          int32_t* trace_slot, int32_t* trace_target, int32_t* trace_u, int32_t* trace_v)
{
    if (n <= 0 || a == NULL || tau_out == NULL || f_out == NULL) return ORACLE_ERR_INVALID;
    if (n > (1 << 17)) return ORACLE_ERR_INVALID;
    if (!oracle_range_ok(a, n)) return ORACLE_ERR_RANGE;

    size_t nb = (size_t)n * sizeof(int32_t);
    int32_t* sigma = (int32_t*)malloc(nb);
    int32_t* tau = (int32_t*)malloc(nb);
    int32_t* dbar = (int32_t*)malloc(nb);   /* delta-bar_i and its job j_i */
    int32_t* jbar = (int32_t*)malloc(nb);
    int32_t* dund = (int32_t*)malloc(nb);   /* delta-underbar_j and its agent i_j */
    int32_t* iund = (int32_t*)malloc(nb);
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    oracle_stats st = {0, 0, 0, 0};
    int status = ORACLE_OK;

    /* Section 3.1: initial solution. */
    if (init_mode == ORACLE_INIT_GREEDY) {
        oracle_greedy_init(a, n, tau);
    } else if (init_mode == ORACLE_INIT_IDENTITY) {
        for (int32_t i = 0; i < n; ++i) tau[i] = i;
    } else if (init_mode == ORACLE_INIT_RANDOM) {
        oracle_random_permutation(n, seed, tau);
    } else if (init_mode == ORACLE_INIT_USER && init_tau != NULL) {
        for (int32_t i = 0; i < n; ++i) {
            if (init_tau[i] < 0 || init_tau[i] >= n || seen[init_tau[i]]) {
                status = ORACLE_ERR_INVALID;
                goto out;
            }
            seen[init_tau[i]] = 1;
            tau[i] = init_tau[i];
        }
    } else {
        status = ORACLE_ERR_INVALID;
        goto out;
    }
    for (int32_t i = 0; i < n; ++i) sigma[tau[i]] = i;
    int64_t f = oracle_objective(a, n, tau);

    for (;;) { /* repeat ... until f(sigma_start) = f(sigma') (R5) */
        st.passes++;
        int64_t f_start = f;
        for (int32_t i = 0; i < n; ++i) oracle_ade(a, n, sigma, tau, i, &dbar[i], &jbar[i]);
        for (int32_t j = 0; j < n; ++j) oracle_jde(a, n, sigma, tau, j, &dund[j], &iund[j]);
        st.evaluations += 2 * (int64_t)n;
        for (;;) { /* switching phase: while some delta > 0 */
            int32_t is = 0, js = 0;
            for (int32_t i = 1; i < n; ++i) if (dbar[i] > dbar[is]) is = i;
            for (int32_t j = 1; j < n; ++j) if (dund[j] > dund[js]) js = j;
            if (dbar[is] <= 0 && dund[js] <= 0) break;
            if (max_iters > 0 && st.sweeps >= max_iters) {
                status = ORACLE_TIMEOUT;
                goto finish;
            }
            int32_t u, v; /* agent u takes the target job, v is the current holder */
            int32_t slot, target;
            if (dbar[is] > dund[js]) {
                dbar[is] = 0;
                slot = is;
                target = jbar[is];
                u = is;
                v = sigma[jbar[is]];
            } else {
                dund[js] = 0;
                slot = n + js;
                target = iund[js];
                u = iund[js];
                v = sigma[js];
            }
            int64_t g = exchange_gain(a, n, tau, u, v);
            int applied = 0;
            if (g > 0) {
                do_exchange(sigma, tau, u, v);
                f += g;
                applied = 1;
                st.swaps_applied++;
                /* the agents and jobs of the exchange: ADE and JDE again */
                oracle_ade(a, n, sigma, tau, u, &dbar[u], &jbar[u]);
                oracle_ade(a, n, sigma, tau, v, &dbar[v], &jbar[v]);
                oracle_jde(a, n, sigma, tau, tau[u], &dund[tau[u]], &iund[tau[u]]);
                oracle_jde(a, n, sigma, tau, tau[v], &dund[tau[v]], &iund[tau[v]]);
                st.evaluations += 4;
            }
            if (st.sweeps < trace_cap) {
                if (trace_applied) trace_applied[st.sweeps] = applied;
                if (trace_objective) trace_objective[st.sweeps] = f;
                if (trace_slot) trace_slot[st.sweeps] = slot;
                if (trace_target) trace_target[st.sweeps] = target;
                if (trace_u) trace_u[st.sweeps] = u;
                if (trace_v) trace_v[st.sweeps] = v;
            }
            st.sweeps++;
        }
        if (f == f_start) break;
    }

finish:
    memcpy(tau_out, tau, nb);
    *f_out = oracle_objective(a, n, tau);
    if (status == ORACLE_OK && *f_out != f) status = ORACLE_ERR_INTERNAL;
out:
    if (stats) *stats = st;
    free(sigma); free(tau); free(dbar); free(jbar); free(dund); free(iund); free(seen);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Rectangular instances (reading R11): the padded square instance. */
int oracle_dgs_rect(const int32_t* a, int32_t n_agents, int32_t m_jobs, int32_t algorithm, int32_t init_mode,
                    uint64_t seed, int32_t reeval_rule, int32_t* assign_out, int64_t* f_out, oracle_stats* stats)
{
    if (a == NULL || assign_out == NULL || f_out == NULL || n_agents <= 0 || m_jobs <= 0) return ORACLE_ERR_INVALID;
    int32_t s = n_agents > m_jobs ? n_agents : m_jobs;
    int32_t* sq = (int32_t*)calloc((size_t)s * s, sizeof(int32_t));
    int32_t* tau = (int32_t*)malloc((size_t)s * sizeof(int32_t));
    for (int32_t i = 0; i < n_agents; ++i)
        memcpy(sq + (size_t)i * s, a + (size_t)i * m_jobs, (size_t)m_jobs * sizeof(int32_t));
    int64_t f = 0;
    int status;
    if (algorithm == 1)
        status = oracle_dgs_sequential(sq, s, init_mode, NULL, seed, 0, tau, &f, stats, 0, NULL, NULL,
                                       NULL, NULL, NULL, NULL);
    else
        status = oracle_dgs_parallel(sq, s, init_mode, NULL, seed, 0, ORACLE_CC_SLOTS, reeval_rule, tau, &f, stats,
                                     0, NULL, NULL, NULL);
    for (int32_t i = 0; i < n_agents; ++i) assign_out[i] = tau[i] < m_jobs ? tau[i] : -1;
    *f_out = f;
    free(sq);
    free(tau);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Exact optimum, Hungarian method (Kuhn 1955) in its shortest augmenting
 * path form: rows are inserted one at a time; a Dijkstra-like scan over
 * reduced costs c[i][j] - u[i] - v[j] (c = -a, minimised) finds the
 * cheapest augmenting path, the potentials are shifted by the scan's
 * minimum at each step and the path is flipped.  1-based internally;
 * column 0 is the virtual root. */
int64_t oracle_hungarian(const int32_t* a, int32_t n, int32_t* tau_out)
{
    const int64_t INF = (int64_t)1 << 62;
    size_t m = (size_t)n + 1;
    int64_t* u = (int64_t*)calloc(m, sizeof(int64_t));
    int64_t* v = (int64_t*)calloc(m, sizeof(int64_t));
    int64_t* min_slack = (int64_t*)malloc(m * sizeof(int64_t));
    int32_t* row_of_col = (int32_t*)calloc(m, sizeof(int32_t));
    int32_t* prev_col = (int32_t*)calloc(m, sizeof(int32_t));
    uint8_t* visited = (uint8_t*)malloc(m);

    for (int32_t r = 1; r <= n; ++r) {
        row_of_col[0] = r;
        int32_t col = 0;
        for (size_t c = 0; c < m; ++c) { min_slack[c] = INF; visited[c] = 0; }
        do {
            visited[col] = 1;
            int32_t row = row_of_col[col];
            int64_t step = INF;
            int32_t next_col = 0;
            for (int32_t c = 1; c <= n; ++c) {
                if (visited[c]) continue;
                int64_t reduced = -A(row - 1, c - 1) - u[row] - v[c];
                if (reduced < min_slack[c]) { min_slack[c] = reduced; prev_col[c] = col; }
                if (min_slack[c] < step) { step = min_slack[c]; next_col = c; }
            }
            for (int32_t c = 0; c <= n; ++c) {
                if (visited[c]) { u[row_of_col[c]] += step; v[c] -= step; }
                else min_slack[c] -= step;
            }
            col = next_col;
        } while (row_of_col[col] != 0);
        do { /* flip the augmenting path back to the root */
            int32_t pc = prev_col[col];
            row_of_col[col] = row_of_col[pc];
            col = pc;
        } while (col != 0);
    }
    for (int32_t c = 1; c <= n; ++c) tau_out[row_of_col[c] - 1] = c - 1;
    free(u); free(v); free(min_slack); free(row_of_col); free(prev_col); free(visited);
    return oracle_objective(a, n, tau_out);
}

/* ------------------------------------------------------------------------ */
/* Exact optimum by enumeration of all permutations in lexicographic order
 * (first optimal permutation kept). */
static void brute_rec(const int32_t* a, int32_t n, int32_t i, int64_t acc,
                      int32_t* cur, uint8_t* used, int64_t* best, int32_t* best_tau)
{
    if (i == n) {
        if (acc > *best) {
            *best = acc;
            memcpy(best_tau, cur, (size_t)n * sizeof(int32_t));
        }
        return;
    }
    for (int32_t j = 0; j < n; ++j) {
        if (used[j]) continue;
        used[j] = 1;
        cur[i] = j;
        brute_rec(a, n, i + 1, acc + A(i, j), cur, used, best, best_tau);
        used[j] = 0;
    }
}

int64_t oracle_brute_force(const int32_t* a, int32_t n, int32_t* tau_out)
{
    int32_t cur[16];
    uint8_t used[16] = {0};
    int64_t best = INT64_MIN;
    if (n > 10) return INT64_MIN;
    brute_rec(a, n, 0, 0, cur, used, &best, tau_out);
    return best;
}
