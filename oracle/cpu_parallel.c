/*
 * cpu_parallel.c -- a second CPU baseline: Algorithm 2's rounds on all host
 * cores (OpenMP), over a worklist of the alive vertices.
 *
 * Test and measurement infrastructure, like the oracle beside it: only the
 * tests and the CPU legs of the benchmark load it, and it shares nothing with
 * the CUDA path.  It is not the oracle: the oracle is the plain sequential
 * restatement in tcmis_oracle.c; this program computes the same rounds
 * (selection test, exclusion test, state update, compaction; Algorithm 2,
 * Sec. 3.1) the way a multicore CPU would, and the tests check that its
 * result, round count and alive sets equal the oracle's.
 *
 * Keys are an input (the oracle's orc_keys gives them), so that the two share
 * one priority definition.  Built with -fopenmp where the compiler has it;
 * without it the pragmas are ignored and it runs on one core.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* u outranks v: larger key, ties to the larger id (as in the oracle). */
static int par_beats(const uint32_t *key, int32_t u, int32_t v)
{
    if (key[u] != key[v]) return key[u] > key[v];
    return u > v;
}

int par_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * status[v] out: 1 = in the MIS.  rounds, alive_sum out; alive_per_round
 * (optional, length >= max_rounds).  threads <= 0: all cores.  Returns 0, or
 * -1 when max_rounds rounds did not empty the alive set or memory ran out.
 */
int par_rounds(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const uint32_t *key,
               uint8_t *status, int32_t *rounds, int64_t *alive_sum, int64_t *alive_per_round,
               int32_t max_rounds, int32_t threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    size_t m = (size_t)(n ? n : 1);
    uint8_t *state = (uint8_t *)malloc(m);     /* 0 undecided, 1 in, 2 out */
    int32_t *wl = (int32_t *)malloc(sizeof(int32_t) * m);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * m);
    uint8_t *cand = (uint8_t *)malloc(m);
    uint8_t *excl = (uint8_t *)malloc(m);
    if (!state || !wl || !next || !cand || !excl) {
        free(state); free(wl); free(next); free(cand); free(excl);
        return -1;
    }
    memset(state, 0, m);
    memset(excl, 0, m);
    for (int32_t v = 0; v < n; ++v) wl[v] = v;
    int64_t len = n, asum = 0;
    int32_t r = 0;
    while (len > 0) {
        if (r >= max_rounds) {
            free(state); free(wl); free(next); free(cand); free(excl);
            return -1;
        }
        if (alive_per_round) alive_per_round[r] = len;
        asum += len;
        /* Phase 1: candidates = alive vertices no alive neighbour outranks */
        #pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < len; ++i) {
            const int32_t v = wl[i];
            int is_max = 1;
            for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
                const int32_t u = col_idx[p];
                if (state[u] == 0 && par_beats(key, u, v)) {
                    is_max = 0;
                    break;
                }
            }
            cand[v] = (uint8_t)is_max;
        }
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < len; ++i)
            if (cand[wl[i]]) state[wl[i]] = 1;
        /* Phase 2: a non-candidate with a candidate neighbour is excluded
           (marked in excl; state is only read here) */
        #pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < len; ++i) {
            const int32_t v = wl[i];
            if (cand[v]) continue;
            for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
                if (cand[col_idx[p]]) {
                    excl[v] = 1;
                    break;
                }
            }
        }
        /* Phase 3: state update, and the rest compacted (in order) into the
           next worklist */
        int64_t k = 0;
        for (int64_t i = 0; i < len; ++i) {
            const int32_t v = wl[i];
            if (excl[v]) state[v] = 2;
            else if (state[v] == 0) next[k++] = v;
            cand[v] = 0;
            excl[v] = 0;
        }
        int32_t *t = wl;
        wl = next;
        next = t;
        len = k;
        ++r;
    }
    for (int32_t v = 0; v < n; ++v) status[v] = state[v] == 1;
    if (rounds) *rounds = r;
    if (alive_sum) *alive_sum = asum;
    free(state); free(wl); free(next); free(cand); free(excl);
    return 0;
}
