/*
 * dgs_oracle.h -- plain CPU oracle for Deep Greedy Switching (single-threaded
 * unless oracle_set_evaluation asks for more threads).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA library.
 *
 * Problem (Section 3, LSAP statement): maximise sum_i a[i][tau(i)] over
 * permutations.  a is n x n, row-major, int32, agent-major (a[i*n + j] is the
 * benefit of giving job j to agent i).  Every entry must satisfy
 * |a| < 2^29 so that every 2-exchange gain (four terms) is exact in int32.
 *
 * Notation (Section 3.3): sigma maps job -> agent, tau = M(sigma) maps
 * agent -> job.  Public outputs are tau (agent -> job).
 *
 * Readings of the paper that this oracle fixes (all listed in the design
 * notes of the repository):
 *   R1 greedy init = global greedy, ties lowest agent then lowest job.
 *   R2 tie-breaks: ADE scans partner jobs ascending with strict '>', so the
 *      lowest job wins; JDE scans partner agents ascending, lowest agent wins;
 *      CC scans slots ascending.
 *   R3 the conflict set C of Algorithm 4 is a set of candidate SLOTS (agent
 *      slots and job slots), partners are looked up in the current sigma.
 *   R4 after the parallel switch, slots not in C are re-evaluated; slots in C
 *      keep their (stale) candidate (the alternative "re-evaluate every
 *      slot" is the option ORACLE_REEVAL_ALL).
 *   R5 the outer repeat stops when a pass leaves f unchanged.
 *
 * Parity: the algorithm is a heuristic, so there is no closed form for its
 * output; the pins are the hand traces, brute force, the Hungarian optimum
 * bound, the local-optimality invariant and the CC characterisation, all in
 * the tests.
 */
#ifndef DGS_ORACLE_H
#define DGS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_INIT_GREEDY = 0, ORACLE_INIT_RANDOM = 1, ORACLE_INIT_IDENTITY = 2, ORACLE_INIT_USER = 3 };
enum { ORACLE_CC_SLOTS = 0, ORACLE_CC_LITERAL_AGENTS = 1 };
enum { ORACLE_REEVAL_BOX = 0, ORACLE_REEVAL_ALL = 1 };
enum { ORACLE_OK = 0, ORACLE_ERR_INVALID = 1, ORACLE_ERR_RANGE = 2, ORACLE_TIMEOUT = 5 };

typedef struct {
    int32_t sweeps;        /* iterations of the switching while-loop (all passes) */
    int32_t passes;        /* iterations of the outer repeat-loop                  */
    int64_t swaps_applied; /* 2-exchanges committed                                */
    int64_t evaluations;   /* single-slot ADE/JDE evaluations performed            */
} oracle_stats;

/* f(tau) = sum_i a[i][tau[i]] in int64 (Section 3 objective). */
int64_t oracle_objective(const int32_t* a, int32_t n, const int32_t* tau);

/* 1 if every |a| < 2^29, else 0. */
int oracle_range_ok(const int32_t* a, int32_t n);

/* Global greedy initial solution (Section 3.1; reading R1). */
void oracle_greedy_init(const int32_t* a, int32_t n, int32_t* tau_out);

/* Random initial solution (Section 3.1, the start the paper itself uses):
 * the identity shuffled by Fisher-Yates in Durstenfeld's form, for i = n-1
 * down to 1 swap positions i and (next() mod (i + 1)), with next() the
 * splitmix64 generator of Steele, Lea and Flood (2014) started at seed. */
void oracle_random_permutation(int32_t n, uint64_t seed, int32_t* tau_out);

/* One step of splitmix64: advances *state and returns the next output. */
uint64_t oracle_splitmix64_next(uint64_t* state);

/* Algorithm 2 (ADE) for agent i: best strictly positive 2-exchange gain and
 * the job it moves agent i to; gain 0 and job -1 when none improves. */
void oracle_ade(const int32_t* a, int32_t n, const int32_t* sigma,
                const int32_t* tau, int32_t i, int32_t* gain, int32_t* job);

/* JDE for job j (Section 3.2): the same exchanges seen from the job, partner
 * agents scanned ascending; gain 0 and agent -1 when none improves. */
void oracle_jde(const int32_t* a, int32_t n, const int32_t* sigma,
                const int32_t* tau, int32_t j, int32_t* gain, int32_t* agent);

/* One fresh difference evaluation of every agent and job (Algorithm 3,
 * first parallel block) for the assignment tau. */
void oracle_evaluate_all(const int32_t* a, int32_t n, const int32_t* tau,
                         int32_t* agent_gain, int32_t* agent_job,
                         int32_t* job_gain, int32_t* job_agent);

/* Algorithm 4 (CC) under reading R3: given the candidate slots and the
 * current sigma, mark conflicted agent slots (in_ca[i] = 1) and conflicted
 * job slots (in_cj[j] = 1).  Slots without a candidate are never in C. */
void oracle_check_conflicts(int32_t n, const int32_t* sigma,
                            const int32_t* agent_gain, const int32_t* agent_job,
                            const int32_t* job_gain, const int32_t* job_agent,
                            uint8_t* in_ca, uint8_t* in_cj);

/* How Algorithm 3's slot evaluations run (process-wide setting): on
 * `threads` host threads (each ADE/JDE writes only its own slot, so the
 * result does not depend on it), and with use_transpose != 0 reading the
 * column entries a[i'][j] from a transposed copy.  Default (1, 0): the
 * literal single-threaded loops. */
void oracle_set_evaluation(int32_t threads, int32_t use_transpose);

/* Algorithm 3 (parallel DGS) to termination or until max_sweeps switching
 * iterations have run (max_sweeps <= 0: no cap).  init_mode is one of
 * ORACLE_INIT_*; init_tau is read only for ORACLE_INIT_USER, seed only for
 * ORACLE_INIT_RANDOM.  cc_rule selects reading R3 (ORACLE_CC_SLOTS) or the
 * literal agent-set C (ORACLE_CC_LITERAL_AGENTS, kept only to show that it
 * never terminates).  reeval_rule selects which slots are re-evaluated after
 * each parallel switch: ORACLE_REEVAL_BOX (reading R4: the slots not in C) or
 * ORACLE_REEVAL_ALL (every slot).
 * Per-sweep trace arrays (may be NULL) receive, for sweep s < trace_cap, the
 * number of accepted candidate slots, the number of committed exchanges and
 * f after the sweep.  Returns ORACLE_OK, ORACLE_TIMEOUT (tau_out and f_out
 * still hold the valid assignment reached), ORACLE_ERR_INVALID or
 * ORACLE_ERR_RANGE. */
int oracle_dgs_parallel(const int32_t* a, int32_t n, int32_t init_mode,
                        const int32_t* init_tau, uint64_t seed, int32_t max_sweeps,
                        int32_t cc_rule, int32_t reeval_rule, int32_t* tau_out, int64_t* f_out,
                        oracle_stats* stats, int32_t trace_cap,
                        int32_t* trace_accepted, int32_t* trace_applied,
                        int64_t* trace_objective);

/* Algorithm 1 (sequential DGS, Section 3.3): after a full difference
 * evaluation, repeatedly take the agent slot with the largest delta-bar and
 * the job slot with the largest delta-underbar (ties: lowest index), keep the
 * agent's candidate if its delta is strictly larger, else the job's; zero
 * that delta; apply the exchange (partner looked up in the current sigma) if
 * it raises f, then re-run ADE for the two agents and JDE for the two jobs it
 * touched (reading R6).  The while loop ends when no delta is positive; the
 * outer repeat (reading R5) re-evaluates everything and runs again until a
 * pass leaves f unchanged.  init_mode / init_tau / seed as for
 * oracle_dgs_parallel; max_iters caps while-loop iterations (<= 0: none).
 * stats->sweeps counts while-loop iterations; trace arrays (may be NULL)
 * receive for iteration s < trace_cap 1/0 for a committed exchange, f, the
 * chosen slot (agent i as i, job j as n + j), its target (job j_i or agent
 * i_j) and the two agents of the exchange examined (u takes the target job,
 * v is that job's holder in the current sigma). */
int oracle_dgs_sequential(const int32_t* a, int32_t n, int32_t init_mode,
                          const int32_t* init_tau, uint64_t seed, int32_t max_iters,
                          int32_t* tau_out, int64_t* f_out, oracle_stats* stats,
                          int32_t trace_cap, int32_t* trace_applied, int64_t* trace_objective,
                          int32_t* trace_slot, int32_t* trace_target, int32_t* trace_u, int32_t* trace_v);

/* Rectangular instances (n_agents x m_jobs, row-major, row = agent): the
 * switching moves an agent to a free job as well as exchanging jobs.  Read
 * (R11) as DGS on the square instance of size max(n, m) padded with
 * zero-benefit dummy agents (n < m) or dummy jobs (n > m), dummies numbered
 * after the real ones: an exchange between a real agent and the dummy holding
 * a free job is exactly the move of that agent to the job (same gain).
 * Options as oracle_dgs_parallel (algorithm 0: Algorithm 3, 1: Algorithm 1).
 * assign_out[i] = job of agent i, or -1 when agent i holds a dummy job;
 * *f_out = sum of the real benefits. */
int oracle_dgs_rect(const int32_t* a, int32_t n_agents, int32_t m_jobs, int32_t algorithm, int32_t init_mode,
                    uint64_t seed, int32_t reeval_rule, int32_t* assign_out, int64_t* f_out, oracle_stats* stats);

/* Exact LSAP maximum by the Hungarian method (Kuhn 1955, in the
 * shortest-augmenting-path form with dual potentials).  O(n^3). */
int64_t oracle_hungarian(const int32_t* a, int32_t n, int32_t* tau_out);

/* Exact LSAP maximum by enumerating all n! permutations (n <= 10). */
int64_t oracle_brute_force(const int32_t* a, int32_t n, int32_t* tau_out);

#ifdef __cplusplus
}
#endif
#endif
