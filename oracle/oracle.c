/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded CPU statement of the temporal path queries that the GPU
 * library answers.  Only the test suite, the smoke check of the package entry point and
 * the CPU-baseline leg of the benchmark load this file; the library never does, and the
 * two share no code.
 *
 * Model (Sec. 2.1): discrete time; an edge (u, v, t, lam) is valid on [t, t + lam], i.e.
 * it departs u at t and arrives at v at t + lam.  All arithmetic is exact uint32.
 * Ordering predicates (Sec. 2.2): consecutive edges A then B form a path when
 * end(A) <= start(B) ("Succeeds", strict = 0) or end(A) < start(B) ("StrictlySucceeds",
 * strict = 1).
 * Window [ta, tw], inclusive at both ends: an edge is usable when t >= ta and
 * t + lam <= tw (the window test of the Update function of Alg. 2, with its first
 * comparison read as "reject t < ta").  The ordering predicate relates consecutive edges
 * only: the first edge of a path may depart at exactly ta and the last may arrive at
 * exactly tw under either predicate.
 *
 * Earliest arrival from s (Alg. 2, read with the source s initialised to ta and the
 * frontier as the set of improved vertices): ea[s] = ta, and for v != s the minimum
 * arrival time over time-respecting paths from s in the window; UNREACHED (0xFFFFFFFF)
 * otherwise.  Latest departure to x (a "minimal temporal path" of Sec. 2.3, defined by
 * the paper's reference on temporal path problems): ld[x] = tw, and for u != x the
 * maximum first departure time over time-respecting paths from u to x in the window;
 * UNREACHED otherwise.
 *
 * Fastest path from s (also a "minimal temporal path" of Sec. 2.3, defined by the same
 * reference): fp[s] = 0, and for v != s the minimum of (arrival - first departure) over
 * time-respecting paths from s to v in the window; UNREACHED otherwise.
 *
 * Shortest duration from s (the reference's "shortest path": least total travel time):
 * sd[s] = 0, and for v != s the minimum of the sum of the edge durations over
 * time-respecting paths from s to v in the window (waiting is free); UNREACHED otherwise.
 * Temporal BFS from s: the least number of edges of such a path (hops[s] = 0).
 *
 * Algorithm: the one-pass scan over the time-ordered edge stream of that reference
 * (credited in Sec. 7): edges are visited in ascending t (descending for latest
 * departure), and every edge sharing the same t is re-swept until nothing changes, which
 * only matters when a zero-duration edge under Succeeds can enable another edge of the
 * same instant.  The time order is a plain stable radix sort of the edge indices.
 */
#include <stdint.h>
#include <stdlib.h>

#define UNREACHED 0xFFFFFFFFu

/* perm[k] = index of the k-th edge in ascending departure time, ties by edge index (the
 * stable order).  A least-significant-digit radix sort of (t, index) pairs: three stable
 * counting passes over 11-bit digits of t, starting from ascending indices, so equal
 * times keep ascending indices.  Requires m < 2^32.  Returns 0, or -1 on bad arguments /
 * allocation failure. */
int oracle_time_order(int64_t m, const uint32_t *t, uint32_t *perm) {
    if (m < 0 || m > (int64_t)0xFFFFFFFFLL || (m > 0 && (!t || !perm))) return -1;
    if (m == 0) return 0;
    uint32_t *idx2 = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    uint32_t *key = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    uint32_t *key2 = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
    int64_t *count = (int64_t *)malloc(2048 * sizeof(int64_t));
    if (!idx2 || !key || !key2 || !count) {
        free(idx2);
        free(key);
        free(key2);
        free(count);
        return -1;
    }
    for (int64_t i = 0; i < m; ++i) {
        perm[i] = (uint32_t)i;
        key[i] = t[i];
    }
    uint32_t *ki = key, *ko = key2, *ii = perm, *io = idx2;
    for (int shift = 0; shift < 33; shift += 11) { /* digits 0-10, 11-21, 22-31 */
        for (int d = 0; d < 2048; ++d) count[d] = 0;
        for (int64_t i = 0; i < m; ++i) ++count[(ki[i] >> shift) & 2047u];
        int64_t run = 0; /* exclusive prefix sums: first slot of each digit */
        for (int d = 0; d < 2048; ++d) {
            int64_t c = count[d];
            count[d] = run;
            run += c;
        }
        for (int64_t i = 0; i < m; ++i) {
            int64_t slot = count[(ki[i] >> shift) & 2047u]++;
            ko[slot] = ki[i];
            io[slot] = ii[i];
        }
        uint32_t *x = ki;
        ki = ko;
        ko = x;
        x = ii;
        ii = io;
        io = x;
    }
    /* after three passes the indices sit in idx2 */
    for (int64_t i = 0; i < m; ++i) perm[i] = ii[i];
    free(idx2);
    free(key);
    free(key2);
    free(count);
    return 0;
}

static int check_common(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                        const uint32_t *lam, const uint32_t *perm, int32_t vtx, uint32_t ta, uint32_t tw,
                        const uint32_t *out) {
    if (n <= 0 || m < 0 || vtx < 0 || vtx >= n || ta > tw || tw > 0xFFFFFFFEu || !out) return -1;
    if (m > 0 && (!src || !dst || !t || !lam || !perm)) return -1;
    return 0;
}

/* Earliest arrival from s within [ta, tw]; out[n]. */
int oracle_earliest_arrival(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                            const uint32_t *lam, const uint32_t *perm, int32_t s, uint32_t ta, uint32_t tw,
                            int strict, uint32_t *out) {
    if (check_common(n, m, src, dst, t, lam, perm, s, ta, tw, out)) return -1;
    for (int64_t v = 0; v < n; ++v) out[v] = UNREACHED;
    out[s] = ta;
    int64_t k = 0;
    while (k < m && t[perm[k]] < ta) ++k; /* edges departing before the window */
    while (k < m && t[perm[k]] <= tw) {
        uint32_t now = t[perm[k]];
        int64_t end = k;
        while (end < m && t[perm[end]] == now) ++end; /* the group of edges departing at `now` */
        int again = 1;
        while (again) {
            again = 0;
            for (int64_t j = k; j < end; ++j) {
                uint32_t e = perm[j];
                uint32_t au = out[src[e]];
                if (au == UNREACHED) continue;                  /* u not reached yet */
                int first = (src[e] == s);                       /* leaves the source */
                if ((strict && !first) ? !(au < now) : !(au <= now)) continue; /* predicate */
                uint64_t arrive = (uint64_t)now + lam[e];
                if (arrive > tw) continue;                      /* leaves the window */
                if (arrive < out[dst[e]]) {
                    out[dst[e]] = (uint32_t)arrive;
                    if (arrive == now && !strict) again = 1;    /* may enable this instant */
                }
            }
        }
        k = end;
    }
    return 0;
}

/* Latest departure towards x within [ta, tw]; out[n]. */
int oracle_latest_departure(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                            const uint32_t *lam, const uint32_t *perm, int32_t x, uint32_t ta, uint32_t tw,
                            int strict, uint32_t *out) {
    if (check_common(n, m, src, dst, t, lam, perm, x, ta, tw, out)) return -1;
    for (int64_t v = 0; v < n; ++v) out[v] = UNREACHED;
    out[x] = tw;
    int64_t k = m - 1;
    while (k >= 0 && t[perm[k]] > tw) --k; /* edges departing after the window */
    while (k >= 0 && t[perm[k]] >= ta) {
        uint32_t now = t[perm[k]];
        int64_t beg = k;
        int has_zero = 0; /* a zero-duration edge of this instant can follow a new label */
        while (beg >= 0 && t[perm[beg]] == now) has_zero |= (lam[perm[beg--]] == 0);
        /* the group is perm[beg+1 .. k] */
        int again = 1;
        while (again) {
            again = 0;
            for (int64_t j = k; j > beg; --j) {
                uint32_t e = perm[j];
                uint32_t lv = out[dst[e]];
                if (lv == UNREACHED) continue;                    /* v cannot reach x */
                uint64_t arrive = (uint64_t)now + lam[e];
                if (arrive > tw) continue;                        /* leaves the window */
                int last = (dst[e] == x);                          /* enters the target */
                if ((strict && !last) ? !(arrive < lv) : !(arrive <= lv)) continue; /* predicate */
                uint32_t lu = out[src[e]];
                if (lu == UNREACHED || now > lu) {
                    out[src[e]] = now; /* u can now be entered by a lam = 0 edge at `now` */
                    if (has_zero && !strict) again = 1;
                }
            }
        }
        k = beg;
    }
    return 0;
}

/* Number of edges usable under final earliest-arrival labels from s: ea[u] reached,
 * t >= ea[u] (> when strict and u != s) and t + lam <= tw.  (t >= ta follows from
 * ea[u] >= ta.) */
uint64_t oracle_admissible_ea(int64_t m, const int32_t *src, const uint32_t *t, const uint32_t *lam,
                              const uint32_t *ea, int32_t s, uint32_t tw, int strict) {
    uint64_t c = 0;
    for (int64_t e = 0; e < m; ++e) {
        uint32_t au = ea[src[e]];
        if (au == UNREACHED) continue;
        if ((strict && src[e] != s) ? !(au < t[e]) : !(au <= t[e])) continue;
        if ((uint64_t)t[e] + lam[e] > tw) continue;
        ++c;
    }
    return c;
}

/* Number of edges usable under final latest-departure labels towards x: ld[v] reached,
 * t + lam <= ld[v] (< when strict and v != x) and t >= ta.  (t + lam <= tw follows from
 * ld[v] <= tw.) */
uint64_t oracle_admissible_ld(int64_t m, const int32_t *dst, const uint32_t *t, const uint32_t *lam,
                              const uint32_t *ld, int32_t x, uint32_t ta, int strict) {
    uint64_t c = 0;
    for (int64_t e = 0; e < m; ++e) {
        uint32_t lv = ld[dst[e]];
        if (lv == UNREACHED) continue;
        uint64_t arrive = (uint64_t)t[e] + lam[e];
        if ((strict && dst[e] != x) ? !(arrive < lv) : !(arrive <= lv)) continue;
        if (t[e] < ta) continue;
        ++c;
    }
    return c;
}

/*
 * Certificate check of a claimed earliest-arrival labelling `ea` at any size, in one pass
 * over the unsorted edges (no sort, O(n + m)).  It holds exactly when `ea` equals the
 * definition above, provided every duration is >= 1 or strict = 1 (then every witness
 * chain strictly decreases in time and ends at s):
 *   (1) ea[s] = ta, and every other reached label lies in (ta, tw];
 *   (2) closure: no usable edge improves a label (ea[u] reached, t >= ea[u] (> when
 *       strict and u != s), t + lam <= tw  =>  ea[v] <= t + lam);
 *   (3) witness: every reached v != s has a usable edge with t + lam == ea[v].
 * (2) gives ea <= EA along every path; (3) with strictly decreasing witness chains gives
 * ea >= EA.  Returns 0 when the certificate holds, 1 when it fails (first offending
 * vertex or edge index in *bad, negative for edges: -(e+1)), -1 on bad arguments,
 * 2 when it does not apply (some lam == 0 with strict == 0).
 */
int oracle_certify_ea(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                      const uint32_t *lam, int32_t s, uint32_t ta, uint32_t tw, int strict,
                      const uint32_t *ea, int64_t *bad) {
    if (n <= 0 || m < 0 || s < 0 || s >= n || ta > tw || !ea || !bad) return -1;
    *bad = 0;
    if (!strict)
        for (int64_t e = 0; e < m; ++e)
            if (lam[e] == 0) return 2;
    if (ea[s] != ta) {
        *bad = s;
        return 1;
    }
    for (int64_t v = 0; v < n; ++v)
        if (v != s && ea[v] != UNREACHED && !(ea[v] > ta && ea[v] <= tw)) {
            *bad = v;
            return 1;
        }
    unsigned char *seen = (unsigned char *)calloc((size_t)n, 1);
    if (!seen) return -1;
    for (int64_t e = 0; e < m; ++e) {
        uint32_t au = ea[src[e]];
        if (au == UNREACHED) continue;
        if ((strict && src[e] != s) ? !(au < t[e]) : !(au <= t[e])) continue;
        uint64_t arrive = (uint64_t)t[e] + lam[e];
        if (arrive > tw) continue;
        if ((uint64_t)ea[dst[e]] > arrive) { /* closure violated */
            free(seen);
            *bad = -(e + 1);
            return 1;
        }
        if ((uint64_t)ea[dst[e]] == arrive) seen[dst[e]] = 1;
    }
    for (int64_t v = 0; v < n; ++v)
        if (v != s && ea[v] != UNREACHED && !seen[v]) { /* no witness */
            free(seen);
            *bad = v;
            return 1;
        }
    free(seen);
    return 0;
}

/*
 * The same certificate for w <= 32 earliest-arrival labellings at once, in one pass over
 * the edges: query q has source s[q], window [ta[q], tw[q]], predicate strict[q] and labels
 * ea[v * w + q] (vertex-major rows, so that the w labels of one vertex are read together).
 * Each query gets the three checks of oracle_certify_ea, independently of the others:
 * status[q] = 0 holds, 1 fails (bad[q] as in oracle_certify_ea), 2 not applicable.
 * Returns 0, or -1 on bad arguments or allocation failure.
 */
int oracle_certify_ea_rows(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                           const uint32_t *lam, int w, const int32_t *s, const uint32_t *ta, const uint32_t *tw,
                           const int32_t *strict, const uint32_t *ea, int32_t *status, int64_t *bad) {
    if (n <= 0 || m < 0 || w < 1 || w > 32 || !s || !ta || !tw || !strict || !ea || !status || !bad) return -1;
    int any_zero = 0;
    for (int64_t e = 0; e < m && !any_zero; ++e) any_zero = lam[e] == 0;
    uint32_t live = 0; /* queries still unrefuted */
    for (int q = 0; q < w; ++q) {
        if (s[q] < 0 || s[q] >= n || ta[q] > tw[q]) return -1;
        status[q] = 0;
        bad[q] = 0;
        if (any_zero && !strict[q]) {
            status[q] = 2;
            continue;
        }
        if (ea[(int64_t)s[q] * w + q] != ta[q]) {
            status[q] = 1;
            bad[q] = s[q];
            continue;
        }
        live |= 1u << q;
    }
    for (int64_t v = 0; v < n; ++v)
        for (int q = 0; q < w; ++q) {
            uint32_t x = ea[v * w + q];
            if (((live >> q) & 1u) && v != s[q] && x != UNREACHED && !(x > ta[q] && x <= tw[q])) {
                status[q] = 1;
                bad[q] = v;
                live &= ~(1u << q);
            }
        }
    uint32_t *seen = (uint32_t *)calloc((size_t)n, sizeof(uint32_t)); /* bit q: v witnessed in query q */
    if (!seen) return -1;
    for (int64_t e = 0; e < m; ++e) {
        const uint32_t *au_row = ea + (int64_t)src[e] * w, *av_row = ea + (int64_t)dst[e] * w;
        for (int q = 0; q < w; ++q) {
            if (!((live >> q) & 1u)) continue;
            uint32_t au = au_row[q];
            if (au == UNREACHED) continue;
            if ((strict[q] && src[e] != s[q]) ? !(au < t[e]) : !(au <= t[e])) continue;
            uint64_t arrive = (uint64_t)t[e] + lam[e];
            if (arrive > tw[q]) continue;
            if ((uint64_t)av_row[q] > arrive) { /* closure violated */
                status[q] = 1;
                bad[q] = -(e + 1);
                live &= ~(1u << q);
                continue;
            }
            if ((uint64_t)av_row[q] == arrive) seen[dst[e]] |= 1u << q;
        }
    }
    for (int64_t v = 0; v < n; ++v)
        for (int q = 0; q < w; ++q)
            if (((live >> q) & 1u) && v != s[q] && ea[v * w + q] != UNREACHED && !((seen[v] >> q) & 1u)) {
                status[q] = 1; /* no witness */
                bad[q] = v;
                live &= ~(1u << q);
            }
    free(seen);
    return 0;
}

/*
 * Fastest paths from s within [ta, tw]; out[n] (durations).  The reference's one-pass
 * fastest-path scan: every vertex v keeps the (start, arrival) pairs of the paths found so
 * far that no other pair dominates (a pair dominates another when it starts no earlier and
 * arrives no later), sorted by start.  Edges are visited in ascending t (equal t re-swept
 * until nothing changes).  An edge (u, v, t, lam) out of s starts a path (t, t + lam); out of
 * another u it extends the pair of u with the latest start among those arriving in time
 * (arrival <= t, < under StrictlySucceeds), which is the pair with the largest such
 * arrival; the result (start, t + lam) joins v's pairs and fp[v] = min(fp[v], t + lam -
 * start).  Pairs are plain arrays grown with realloc and kept sorted by insertion.
 */
typedef struct {
    uint32_t *s, *a; /* starts ascending, arrivals ascending */
    int64_t len, cap;
} pair_list;

/* Insert (s, a) unless a pair dominates it; drop the pairs it dominates.  Returns 1 when
 * the list changed, 0 when not, -1 on allocation failure. */
static int pairs_insert(pair_list *L, uint32_t s, uint32_t a) {
    for (int64_t i = 0; i < L->len; ++i)
        if (L->s[i] >= s && L->a[i] <= a) return 0; /* dominated */
    int64_t w = 0;
    for (int64_t i = 0; i < L->len; ++i)
        if (!(L->s[i] <= s && L->a[i] >= a)) { /* keep what the new pair does not dominate */
            L->s[w] = L->s[i];
            L->a[w] = L->a[i];
            ++w;
        }
    L->len = w;
    if (L->len == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 4;
        uint32_t *ns = (uint32_t *)realloc(L->s, (size_t)nc * sizeof(uint32_t));
        if (!ns) return -1;
        L->s = ns;
        uint32_t *na = (uint32_t *)realloc(L->a, (size_t)nc * sizeof(uint32_t));
        if (!na) return -1;
        L->a = na;
        L->cap = nc;
    }
    int64_t p = L->len; /* sorted position by start */
    while (p > 0 && L->s[p - 1] > s) {
        L->s[p] = L->s[p - 1];
        L->a[p] = L->a[p - 1];
        --p;
    }
    L->s[p] = s;
    L->a[p] = a;
    ++L->len;
    return 1;
}

int oracle_fastest(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                   const uint32_t *lam, const uint32_t *perm, int32_t s, uint32_t ta, uint32_t tw, int strict,
                   uint32_t *out) {
    if (check_common(n, m, src, dst, t, lam, perm, s, ta, tw, out)) return -1;
    pair_list *P = (pair_list *)calloc((size_t)n, sizeof(pair_list));
    uint64_t *best = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int rc = 0;
    if (!P || !best) {
        rc = -1;
        goto done;
    }
    for (int64_t v = 0; v < n; ++v) best[v] = UINT64_MAX;
    best[s] = 0;
    int64_t k = 0;
    while (k < m && t[perm[k]] < ta) ++k; /* edges departing before the window */
    while (k < m && t[perm[k]] <= tw) {
        uint32_t now = t[perm[k]];
        int64_t end = k;
        while (end < m && t[perm[end]] == now) ++end;
        int again = 1;
        while (again) {
            again = 0;
            for (int64_t j = k; j < end; ++j) {
                uint32_t e = perm[j];
                uint64_t arrive = (uint64_t)now + lam[e];
                if (arrive > tw) continue; /* leaves the window */
                int32_t u = src[e], v = dst[e];
                if (v == s) continue; /* a path back to s never beats fp[s] = 0 or a fresh start */
                uint32_t start;
                if (u == s) {
                    start = now; /* depart s now: no later start exists for this edge */
                } else {
                    const pair_list *L = &P[u];
                    int64_t i = L->len - 1; /* largest arrival that is in time */
                    while (i >= 0 && (strict ? !(L->a[i] < now) : !(L->a[i] <= now))) --i;
                    if (i < 0) continue; /* u not reached in time */
                    start = L->s[i];
                }
                int ch = pairs_insert(&P[v], start, (uint32_t)arrive);
                if (ch < 0) {
                    rc = -1;
                    goto done;
                }
                if (ch) {
                    if (arrive - start < best[v]) best[v] = arrive - start;
                    again = 1; /* a new pair may enable another edge of this instant */
                }
            }
        }
        k = end;
    }
    for (int64_t v = 0; v < n; ++v) out[v] = best[v] == UINT64_MAX ? UNREACHED : (uint32_t)best[v];
done:
    if (P) {
        for (int64_t v = 0; v < n; ++v) {
            free(P[v].s);
            free(P[v].a);
        }
        free(P);
    }
    free(best);
    return rc;
}

/*
 * Shortest durations from s within [ta, tw]; out[n].  The reference's one-pass
 * shortest-path scan: every vertex v keeps the (total duration, arrival) pairs of the paths
 * found so far that no other pair dominates (a pair dominates another when its total is no
 * larger and it arrives no later), sorted by arrival (totals then strictly decrease).
 * Edges are visited in ascending t (equal t re-swept until nothing changes).  An edge
 * (u, v, t, lam) out of s starts a path (lam, t + lam); out of another u it extends the
 * pair of u with the smallest total among those arriving in time (arrival <= t, < under
 * StrictlySucceeds), which is the in-time pair with the latest arrival; the result
 * (total + lam, t + lam) joins v's pairs and sd[v] = min(sd[v], total + lam).
 */
static int dpairs_insert(pair_list *L, uint32_t d, uint32_t a) {
    /* here pair_list.s holds totals, .a arrivals; sorted by arrival ascending */
    for (int64_t i = 0; i < L->len; ++i)
        if (L->s[i] <= d && L->a[i] <= a) return 0; /* dominated */
    int64_t w = 0;
    for (int64_t i = 0; i < L->len; ++i)
        if (!(L->s[i] >= d && L->a[i] >= a)) {
            L->s[w] = L->s[i];
            L->a[w] = L->a[i];
            ++w;
        }
    L->len = w;
    if (L->len == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 4;
        uint32_t *ns = (uint32_t *)realloc(L->s, (size_t)nc * sizeof(uint32_t));
        if (!ns) return -1;
        L->s = ns;
        uint32_t *na = (uint32_t *)realloc(L->a, (size_t)nc * sizeof(uint32_t));
        if (!na) return -1;
        L->a = na;
        L->cap = nc;
    }
    int64_t p = L->len; /* sorted position by arrival */
    while (p > 0 && L->a[p - 1] > a) {
        L->s[p] = L->s[p - 1];
        L->a[p] = L->a[p - 1];
        --p;
    }
    L->s[p] = d;
    L->a[p] = a;
    ++L->len;
    return 1;
}

/* cost of an edge: its duration, or 1 (unit = 1: temporal BFS, the least number of edges) */
static int least_cost_scan(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                           const uint32_t *lam, const uint32_t *perm, int32_t s, uint32_t ta, uint32_t tw, int strict,
                           int unit, uint32_t *out) {
    if (check_common(n, m, src, dst, t, lam, perm, s, ta, tw, out)) return -1;
    pair_list *P = (pair_list *)calloc((size_t)n, sizeof(pair_list));
    uint64_t *best = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int rc = 0;
    if (!P || !best) {
        rc = -1;
        goto done;
    }
    for (int64_t v = 0; v < n; ++v) best[v] = UINT64_MAX;
    best[s] = 0;
    int64_t k = 0;
    while (k < m && t[perm[k]] < ta) ++k; /* edges departing before the window */
    while (k < m && t[perm[k]] <= tw) {
        uint32_t now = t[perm[k]];
        int64_t end = k;
        while (end < m && t[perm[end]] == now) ++end;
        int again = 1;
        while (again) {
            again = 0;
            for (int64_t j = k; j < end; ++j) {
                uint32_t e = perm[j];
                uint64_t arrive = (uint64_t)now + lam[e];
                if (arrive > tw) continue; /* leaves the window */
                int32_t u = src[e], v = dst[e];
                if (v == s) continue; /* nothing beats sd[s] = 0 or a fresh start */
                uint64_t base;
                if (u == s) {
                    base = 0;
                } else {
                    const pair_list *L = &P[u];
                    int64_t i = L->len - 1; /* latest arrival in time = smallest total */
                    while (i >= 0 && (strict ? !(L->a[i] < now) : !(L->a[i] <= now))) --i;
                    if (i < 0) continue;
                    base = L->s[i];
                }
                uint64_t total = base + (unit ? 1u : lam[e]);
                if (total > 0xFFFFFFFEu) continue; /* beyond any label (cannot happen for usable edges) */
                int ch = dpairs_insert(&P[v], (uint32_t)total, (uint32_t)arrive);
                if (ch < 0) {
                    rc = -1;
                    goto done;
                }
                if (ch) {
                    if (total < best[v]) best[v] = total;
                    again = 1;
                }
            }
        }
        k = end;
    }
    for (int64_t v = 0; v < n; ++v) out[v] = best[v] == UINT64_MAX ? UNREACHED : (uint32_t)best[v];
done:
    if (P) {
        for (int64_t v = 0; v < n; ++v) {
            free(P[v].s);
            free(P[v].a);
        }
        free(P);
    }
    free(best);
    return rc;
}

int oracle_shortest_duration(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                             const uint32_t *lam, const uint32_t *perm, int32_t s, uint32_t ta, uint32_t tw,
                             int strict, uint32_t *out) {
    return least_cost_scan(n, m, src, dst, t, lam, perm, s, ta, tw, strict, 0, out);
}

/*
 * Temporal BFS from s within [ta, tw]: out[v] = the least number of edges of a
 * time-respecting path from s to v in the window (out[s] = 0), UNREACHED otherwise.  The same
 * pair scan as shortest durations with every edge costing 1.
 */
int oracle_temporal_bfs(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                        const uint32_t *lam, const uint32_t *perm, int32_t s, uint32_t ta, uint32_t tw, int strict,
                        uint32_t *out) {
    return least_cost_scan(n, m, src, dst, t, lam, perm, s, ta, tw, strict, 1, out);
}

/*
 * Temporal connected components within [ta, tw] (the connectivity application of Sec. 2.3 and
 * Table 4, "adapted to accept a start and end time" as Sec. 6 describes): the connected
 * components of the undirected graph formed by the edges usable in the window (t >= ta and
 * t + lam <= tw), every vertex included.  out[v] = the smallest vertex id of v's component (a
 * vertex with no usable edge is its own component).  A plain union-find: every usable edge
 * unites its endpoints (the root is the smaller id, found by following parents with path
 * halving); then each vertex takes its root.  Returns 0, or -1 on bad arguments / allocation.
 */
static int32_t uf_find(int32_t *parent, int32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

int oracle_temporal_cc(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, const uint32_t *t,
                       const uint32_t *lam, uint32_t ta, uint32_t tw, uint32_t *out) {
    if (n <= 0 || m < 0 || ta > tw || !out || (m > 0 && (!src || !dst || !t || !lam))) return -1;
    int32_t *parent = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!parent) return -1;
    for (int64_t v = 0; v < n; ++v) parent[v] = (int32_t)v;
    for (int64_t e = 0; e < m; ++e) {
        if (t[e] < ta || (uint64_t)t[e] + lam[e] > tw) continue; /* not usable in the window */
        int32_t a = uf_find(parent, src[e]), b = uf_find(parent, dst[e]);
        if (a == b) continue;
        if (a < b) parent[b] = a; else parent[a] = b; /* the smaller id stays the root */
    }
    for (int64_t v = 0; v < n; ++v) out[v] = (uint32_t)uf_find(parent, (int32_t)v);
    free(parent);
    return 0;
}
