/*
 * tcmis_oracle.c -- CPU oracle for the TC-MIS hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it; the library's own
 * code path never does.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Contents, each following the paper (TC-MIS, Nijhara & Banerjee):
 *
 *   orc_keys         Eq. 1 degree-aware priority P(v) = d / (d + deg(v) - eps(v)),
 *                    d = average degree, eps a small hashed perturbation
 *                    (Sec. 2, Eq. 1; Sec. 3.3 H2).  Priorities are assigned once
 *                    and reused every round (Sec. 2, random-permutation variant).
 *   orc_keys_mode    the keys of the other priority heuristics of Sec. 3.3: H1
 *                    (random, hash(v)) and Eq. 1 discretised to 8 bits.
 *   orc_rounds       Algorithm 2 (and Algorithm 1): while the alive set A is not
 *                    empty -- Phase 1 candidates C = strict local maxima of P among
 *                    alive neighbours; Phase 2 N_c = A x C (neighbour counts of
 *                    candidates); Phase 3 M += C, A -= C and every v with
 *                    N_c(v) > 0.  Every quantity of one round is computed from the
 *                    round-start snapshot (the H3 ordering of Sec. 3.3).
 *   orc_greedy       the closed form of the same result: sequential greedy in
 *                    decreasing priority order (the lexicographically-first MIS;
 *                    Blelloch, Fineman, Shun, SPAA 2012).
 *   orc_min_degree_greedy  quality yardstick (not parity): dynamic min-degree greedy.
 *   orc_check        independence and maximality of a result.
 *
 * Readings of points the paper leaves open (each one also listed in the design
 * notes of the repository):
 *   - d = arcs / n, with arcs = row_ptr[n] (both directions counted), computed
 *     in binary32 as float(arcs) / float(n), round-to-nearest.
 *   - eps(v) = (h >> 8) * 2^-24 with h the high 32 bits of
 *     mix64(mix64(seed) XOR v), mix64 the splitmix64 finaliser
 *     (Steele, Lea, Flood, OOPSLA 2014); eps in [0, 1).
 *   - P is evaluated in binary32, round-to-nearest, as
 *     den = (d + float(deg)) - eps; P = d / den; the priority key is the bit
 *     pattern of P (order-preserving because P > 0).  An isolated vertex gets
 *     key 0xFFFFFFFF (it has no neighbour to compare against).
 *   - Ties in P are broken by vertex id, the larger id winning: the order is
 *     lexicographic on (key, id).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math (no FMA
 * contraction, IEEE binary32 arithmetic for every float operation).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* splitmix64 finaliser (Steele, Lea, Flood 2014). */
static uint64_t orc_mix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ULL;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return z;
}

uint64_t orc_splitmix64_mix(uint64_t z) { return orc_mix64(z); }

/* The hashed perturbation eps(v) of Eq. 1, as an exact binary32 in [0, 1). */
float orc_eps(uint64_t seed, int32_t local_id)
{
    uint64_t h64 = orc_mix64(orc_mix64(seed) ^ (uint64_t)(uint32_t)local_id);
    uint32_t h = (uint32_t)(h64 >> 32);
    return (float)(h >> 8) * 0x1p-24f;
}

/* Eq. 1 for one vertex: P = dbar / (dbar + deg - eps), binary32 RN. */
float orc_priority(float dbar, int32_t deg, float eps)
{
    float den = dbar + (float)deg;
    den = den - eps;
    return dbar / den;
}

static uint32_t orc_float_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

/*
 * Priority keys of one graph (Eq. 1; assigned once per solve, Sec. 2).
 * key[v] = bits of P(v) for deg(v) >= 1, 0xFFFFFFFF for deg(v) = 0.
 * v is the vertex id within its own graph.
 */
void orc_keys(int32_t n, const int32_t *row_ptr, uint64_t seed, uint32_t *key)
{
    if (n <= 0) return;
    float dbar = (float)row_ptr[n] / (float)n;
    for (int32_t v = 0; v < n; ++v) {
        int32_t deg = row_ptr[v + 1] - row_ptr[v];
        if (deg == 0) {
            key[v] = 0xFFFFFFFFu;
            continue;
        }
        float p = orc_priority(dbar, deg, orc_eps(seed, v));
        key[v] = orc_float_bits(p);
    }
}

/*
 * Priority keys under one of the paper's priority heuristics (Sec. 3.3):
 *   mode 0  H2 / H3, the degree-aware Eq. 1: exactly orc_keys;
 *   mode 1  H1, random priority P(v) = hash(v): the high 29 bits of
 *           h = hi32(mix64(mix64(seed) XOR v)), written as 2^29 + (h >> 3);
 *   mode 2  Eq. 1 scaled and discretised to a compact 8-bit integer (Sec. 2:
 *           the value is scaled and discretized for GPU execution):
 *           q = trunc(P * 255) with P the binary32 Eq. 1 value and the product
 *           in binary32 round-to-nearest; key = q in [0, 255].
 * Isolated vertices get 0xFFFFFFFF in every mode; ties are broken by id as
 * in orc_rounds (they are frequent in mode 2).
 */
void orc_keys_mode(int32_t n, const int32_t *row_ptr, uint64_t seed, int32_t mode, uint32_t *key)
{
    if (n <= 0) return;
    float dbar = (float)row_ptr[n] / (float)n;
    for (int32_t v = 0; v < n; ++v) {
        int32_t deg = row_ptr[v + 1] - row_ptr[v];
        if (deg == 0) {
            key[v] = 0xFFFFFFFFu;
            continue;
        }
        if (mode == 1) {
            uint32_t h = (uint32_t)(orc_mix64(orc_mix64(seed) ^ (uint64_t)(uint32_t)v) >> 32);
            key[v] = 0x20000000u + (h >> 3);
        } else if (mode == 2) {
            float p = orc_priority(dbar, deg, orc_eps(seed, v));
            float scaled = p * 255.0f;
            key[v] = (uint32_t)scaled; /* truncation toward zero; scaled in [0, 255] */
        } else {
            key[v] = orc_float_bits(orc_priority(dbar, deg, orc_eps(seed, v)));
        }
    }
}

/* (key(u), u) precedes-or-beats (key(v), v): larger key wins, then larger id. */
static int orc_beats(const uint32_t *key, int32_t u, int32_t v)
{
    if (key[u] != key[v]) return key[u] > key[v];
    return u > v;
}

/*
 * Algorithm 2, round by round, from the round-start snapshot.
 *   status[v] out: 1 = in the MIS, 0 = not.
 *   rounds   out: number of while-loop iterations (alive set non-empty).
 *   work     out: sum over rounds of the degrees of the vertices alive at the
 *                 round start (the arcs a full pull scan of the alive rows reads).
 *   alive_sum out: sum over rounds of the alive-set size at the round start.
 *   alive_per_round (optional, length >= max_rounds): alive-set size at the
 *                 start of each round.
 * Returns 0, or -1 if `max_rounds` rounds did not empty the alive set or
 * memory ran out.
 */
int orc_rounds(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const uint32_t *key,
               uint8_t *status, int32_t *rounds, int64_t *work, int64_t *alive_sum,
               int64_t *alive_per_round, int32_t max_rounds)
{
    uint8_t *alive = (uint8_t *)malloc((size_t)(n ? n : 1));
    uint8_t *cand = (uint8_t *)malloc((size_t)(n ? n : 1));
    int32_t *nc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    if (!alive || !cand || !nc) {
        free(alive);
        free(cand);
        free(nc);
        return -1;
    }
    int64_t n_alive = n, w = 0, asum = 0;
    int32_t r = 0;
    for (int32_t v = 0; v < n; ++v) {
        alive[v] = 1;
        status[v] = 0;
    }
    while (n_alive > 0) {
        if (r >= max_rounds) {
            free(alive);
            free(cand);
            free(nc);
            return -1;
        }
        if (alive_per_round) alive_per_round[r] = n_alive;
        asum += n_alive;
        /* Phase 1: Max_Np(v) over alive neighbours; C(v) = [P(v) > Max_Np(v)] */
        for (int32_t v = 0; v < n; ++v) {
            cand[v] = 0;
            if (!alive[v]) continue;
            w += row_ptr[v + 1] - row_ptr[v];
            int is_max = 1;
            for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
                int32_t u = col_idx[p];
                if (alive[u] && orc_beats(key, u, v)) {
                    is_max = 0;
                    break;
                }
            }
            cand[v] = (uint8_t)is_max;
        }
        /* Phase 2: N_c = A x C (number of candidate neighbours) */
        for (int32_t v = 0; v < n; ++v) {
            int32_t s = 0;
            for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) s += cand[col_idx[p]];
            nc[v] = s;
        }
        /* Phase 3: M += C; A -= {v : C(v) = 1 or N_c(v) > 0} */
        for (int32_t v = 0; v < n; ++v) {
            if (!alive[v]) continue;
            if (cand[v]) {
                status[v] = 1;
                alive[v] = 0;
                --n_alive;
            } else if (nc[v] > 0) {
                alive[v] = 0;
                --n_alive;
            }
        }
        ++r;
    }
    if (rounds) *rounds = r;
    if (work) *work = w;
    if (alive_sum) *alive_sum = asum;
    free(alive);
    free(cand);
    free(nc);
    return 0;
}

/* sort helper for orc_greedy: decreasing (key, id) */
static const uint32_t *orc_sort_key;
static int orc_cmp_desc(const void *a, const void *b)
{
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    if (orc_sort_key[u] != orc_sort_key[v]) return orc_sort_key[u] > orc_sort_key[v] ? -1 : 1;
    return u > v ? -1 : (u < v);
}

/*
 * Sequential greedy in decreasing (key, id) order: take v iff no neighbour
 * was taken before.  With fixed, strictly ordered priorities this is the
 * unique set the round iteration of Algorithm 2 converges to.
 */
int orc_greedy(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const uint32_t *key,
               uint8_t *status)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    if (!order) return -1;
    for (int32_t v = 0; v < n; ++v) {
        order[v] = v;
        status[v] = 0;
    }
    orc_sort_key = key;
    qsort(order, (size_t)n, sizeof(int32_t), orc_cmp_desc);
    for (int32_t i = 0; i < n; ++i) {
        int32_t v = order[i], ok = 1;
        for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p)
            if (status[col_idx[p]]) {
                ok = 0;
                break;
            }
        status[v] = (uint8_t)ok;
    }
    free(order);
    return 0;
}

/*
 * Independence and maximality of status[] (1 = in the set).
 * Returns 0 if both hold, 1 if two adjacent vertices are in the set, 2 if a
 * vertex outside the set has no neighbour in it.  *bad receives the vertex.
 */
int orc_check(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const uint8_t *status,
              int32_t *bad)
{
    for (int32_t v = 0; v < n; ++v) {
        int covered = status[v] != 0;
        for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
            int32_t u = col_idx[p];
            if (status[v] && status[u]) {
                if (bad) *bad = v;
                return 1;
            }
            if (status[u]) covered = 1;
        }
        if (!covered) {
            if (bad) *bad = v;
            return 2;
        }
    }
    return 0;
}

/*
 * Dynamic min-degree greedy (quality yardstick only): repeatedly take a
 * vertex of minimum remaining degree, delete it and its neighbours, update
 * remaining degrees.  Bucket queue (stacks) with lazy deletion; ties go to
 * the most recently queued vertex.
 * Returns the set size, or -1 on allocation failure.
 */
int64_t orc_min_degree_greedy(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                              uint8_t *status)
{
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    uint8_t *gone = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    int32_t maxd = 0;
    if (!deg || !gone) {
        free(deg);
        free(gone);
        return -1;
    }
    for (int32_t v = 0; v < n; ++v) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        if (deg[v] > maxd) maxd = deg[v];
        status[v] = 0;
    }
    /* bucket lists as singly linked stacks; stale entries skipped lazily */
    int64_t cap = (int64_t)n + (int64_t)row_ptr[n] + 1;
    int32_t *head = (int32_t *)malloc(sizeof(int32_t) * ((size_t)maxd + 1));
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *who = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *bdeg = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!head || !nxt || !who || !bdeg) {
        free(deg);
        free(gone);
        free(head);
        free(nxt);
        free(who);
        free(bdeg);
        return -1;
    }
    for (int32_t d = 0; d <= maxd; ++d) head[d] = -1;
    int64_t used = 0;
    for (int32_t v = n - 1; v >= 0; --v) {
        who[used] = v;
        bdeg[used] = deg[v];
        nxt[used] = head[deg[v]];
        head[deg[v]] = (int32_t)used;
        ++used;
    }
    int64_t size = 0;
    int32_t d = 0;
    while (d <= maxd) {
        int32_t e = head[d];
        if (e < 0) {
            ++d;
            continue;
        }
        head[d] = nxt[e];
        int32_t v = who[e];
        if (gone[v] || bdeg[e] != deg[v]) continue; /* stale */
        status[v] = 1;
        ++size;
        gone[v] = 1;
        for (int32_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
            int32_t u = col_idx[p];
            if (gone[u]) continue;
            gone[u] = 1;
            for (int32_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q) {
                int32_t x = col_idx[q];
                if (gone[x]) continue;
                int32_t nd = --deg[x];
                if (used < cap) {
                    who[used] = x;
                    bdeg[used] = nd;
                    nxt[used] = head[nd];
                    head[nd] = (int32_t)used;
                    ++used;
                }
                if (nd < d) d = nd;
            }
        }
    }
    free(deg);
    free(gone);
    free(head);
    free(nxt);
    free(who);
    free(bdeg);
    return size;
}
