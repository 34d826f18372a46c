/*
 * oracle.c -- plain, slow, sequential CPU statement of what the co-rank /
 * stable-merge path computes (Siebert & Traeff, "Perfectly load-balanced,
 * optimal, stable, parallel merge").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no header, helper, table
 * or constant with the CUDA path.
 *
 * Notation follows the paper: output rank i, co-ranks j (into A) and k (into
 * B), with j + k = i.  Keys are compared with the natural order of their C
 * type (signed for int32/int64, unsigned for uint32/uint64).
 *
 * Functions (one copy per key type, generated by ORC_DEFINE below):
 *   orc_co_rank_T       Algorithm 1 (Section 2), literally, with a trace.
 *   orc_merge_T         sequential stable two-way merge (Section 1 and the
 *                       stability definition of Section 2): ties take A.
 *   orc_merge_kv_T      the same merge carrying a payload of vb bytes (bit copy).
 *   orc_merge_grad_T    gradient of the key-value merge w.r.t. the payloads:
 *                       gA[j] = gC[pos of A[j] in C], gB[k] likewise.
 *   orc_batched_merge_kv_T / orc_batched_merge_grad_T
 *                       the key-value merge applied to every segment pair.
 *   orc_merge_pass_T    one pass of a bottom-up merge sort: adjacent runs of
 *                       width w merged pairwise.
 *   orc_parallel_merge_T Algorithm 2 (Section 3) on p POSIX threads.
 *
 * Build: gcc -O2 -shared -fPIC -pthread oracle.c -o liboracle.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

static int64_t orc_min64(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t orc_max64(int64_t a, int64_t b) { return a > b ? a : b; }

#define ORC_DEFINE(SUF, T)                                                     \
                                                                               \
/* Algorithm 1 (Section 2): co_rank(i, A, m, B, n).                            \
 * Starts from j = min(i, m), k = i - j, j_low = max(0, i - n) and halves      \
 * the interval [j_low, j] (first Lemma condition violated) or [k_low, k]      \
 * (second Lemma condition violated) until both conditions of Lemma 1 hold.    \
 * The "conditional and" of the paper is C's &&.  The paper leaves k_low       \
 * unset before the loop; it argues that only the first condition can fail    \
 * in the first iteration, so k_low is always written before it is read.       \
 * Here k_low carries a "set" flag and the call returns -2 if that argument    \
 * were ever wrong (the second condition failing with k_low unset).            \
 * trace (nullable): 5 int64 per state -- j, k, j_low, k_low (-1 = unset),     \
 * branch (0 = start, 1 = first condition violated, 2 = second) -- for the     \
 * start state and after every iteration that moved (j, k); at most           \
 * trace_cap states are written.  Returns the number of moving iterations,     \
 * -1 if i is outside [0, m+n].                                                \
 * Range: Lemma 1 states 0 <= i < m+n; Proposition 1 and Algorithm 2 use       \
 * i = m+n as well, which is accepted here (result (m, n)).  */                \
int64_t orc_co_rank_##SUF(const T* A, int64_t m, const T* B, int64_t n,        \
                          int64_t i, int64_t* j_out, int64_t* k_out,           \
                          int64_t* trace, int64_t trace_cap)                   \
{                                                                              \
    if (i < 0 || i > m + n) return -1;                                         \
    int64_t j = orc_min64(i, m);                                               \
    int64_t k = i - j;                                                         \
    int64_t j_low = orc_max64(0, i - n);                                       \
    int64_t k_low = 0;                                                         \
    int k_low_set = 0;                                                         \
    int64_t delta;                                                             \
    int64_t moves = 0, nt = 0;                                                 \
    int active = 1;                                                            \
    if (trace && nt < trace_cap) {                                             \
        trace[5*nt+0] = j; trace[5*nt+1] = k; trace[5*nt+2] = j_low;           \
        trace[5*nt+3] = -1; trace[5*nt+4] = 0; nt++;                           \
    }                                                                          \
    while (active) {                                                           \
        if (j > 0 && k < n && A[j-1] > B[k]) {                                 \
            /* first Lemma condition violated: j too large */                  \
            delta = (j - j_low + 1) / 2;                                       \
            k_low = k; k_low_set = 1;                                          \
            j = j - delta; k = k + delta;                                      \
            moves++;                                                           \
            if (trace && nt < trace_cap) {                                     \
                trace[5*nt+0] = j; trace[5*nt+1] = k; trace[5*nt+2] = j_low;   \
                trace[5*nt+3] = k_low; trace[5*nt+4] = 1; nt++;                \
            }                                                                  \
        } else if (k > 0 && j < m && B[k-1] >= A[j]) {                         \
            /* second Lemma condition violated: k too large */                 \
            if (!k_low_set) return -2;                                         \
            delta = (k - k_low + 1) / 2;                                       \
            j_low = j;                                                         \
            j = j + delta; k = k - delta;                                      \
            moves++;                                                           \
            if (trace && nt < trace_cap) {                                     \
                trace[5*nt+0] = j; trace[5*nt+1] = k; trace[5*nt+2] = j_low;   \
                trace[5*nt+3] = k_low; trace[5*nt+4] = 2; nt++;                \
            }                                                                  \
        } else {                                                               \
            active = 0;                                                        \
        }                                                                      \
    }                                                                          \
    *j_out = j; *k_out = k;                                                    \
    return moves;                                                              \
}                                                                              \
                                                                               \
/* co_rank for cnt output ranks (each by Algorithm 1); j = k = -1 for a rank   \
 * outside [0, m+n]. */                                                        \
void orc_co_rank_many_##SUF(const T* A, int64_t m, const T* B, int64_t n,      \
                            const int64_t* ranks, int64_t cnt,                 \
                            int64_t* j_out, int64_t* k_out)                    \
{                                                                              \
    for (int64_t q = 0; q < cnt; ++q) {                                        \
        if (orc_co_rank_##SUF(A, m, B, n, ranks[q], &j_out[q], &k_out[q],      \
                              0, 0) < 0) { j_out[q] = -1; k_out[q] = -1; }     \
    }                                                                          \
}                                                                              \
                                                                               \
/* Sequential stable two-way merge (Section 1; stability as defined in         \
 * Section 2: equal keys keep their order inside A and inside B, and every     \
 * A element precedes an equal B element).  B[k] is taken only when it is      \
 * strictly smaller than A[j].  src (nullable) receives, for every output      \
 * position, the input position: j for A[j], m + k for B[k]. */               \
void orc_merge_##SUF(const T* A, int64_t m, const T* B, int64_t n,             \
                     T* C, int64_t* src)                                       \
{                                                                              \
    int64_t j = 0, k = 0, i = 0;                                               \
    while (j < m && k < n) {                                                   \
        if (B[k] < A[j]) { C[i] = B[k]; if (src) src[i] = m + k; k++; }        \
        else             { C[i] = A[j]; if (src) src[i] = j;     j++; }        \
        i++;                                                                   \
    }                                                                          \
    while (j < m) { C[i] = A[j]; if (src) src[i] = j;     j++; i++; }          \
    while (k < n) { C[i] = B[k]; if (src) src[i] = m + k; k++; i++; }          \
}                                                                              \
                                                                               \
/* Key-value merge: the payload of every element (vb bytes) moves with its    \
 * key, copied bit for bit.  src as in orc_merge (nullable). */                \
int orc_merge_kv_##SUF(const T* A, const void* Av, int64_t m,                  \
                       const T* B, const void* Bv, int64_t n, int64_t vb,      \
                       T* C, void* Cv, int64_t* src)                           \
{                                                                              \
    int64_t* s = src ? src : (int64_t*)malloc(sizeof(int64_t) * (m + n + 1));  \
    if (!s) return -1;                                                         \
    orc_merge_##SUF(A, m, B, n, C, s);                                         \
    for (int64_t i = 0; i < m + n; ++i) {                                      \
        const char* from = s[i] < m ? (const char*)Av + vb * s[i]              \
                                    : (const char*)Bv + vb * (s[i] - m);       \
        memcpy((char*)Cv + vb * i, from, (size_t)vb);                          \
    }                                                                          \
    if (!src) free(s);                                                         \
    return 0;                                                                  \
}                                                                              \
                                                                               \
/* Gradient of C_v = merge_kv(A, Av, B, Bv).v with respect to Av and Bv.       \
 * The merge is a permutation of the payloads, so the gradient routes          \
 * gC[i] back to the input position the element came from (bit copy). */      \
int orc_merge_grad_##SUF(const T* A, int64_t m, const T* B, int64_t n,         \
                         const void* gC, int64_t vb, void* gA, void* gB)       \
{                                                                              \
    int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (m + n + 1));              \
    T* C = (T*)malloc(sizeof(T) * (m + n + 1));                                \
    if (!s || !C) { free(s); free(C); return -1; }                             \
    orc_merge_##SUF(A, m, B, n, C, s);                                         \
    for (int64_t i = 0; i < m + n; ++i) {                                      \
        char* to = s[i] < m ? (char*)gA + vb * s[i]                            \
                            : (char*)gB + vb * (s[i] - m);                     \
        memcpy(to, (const char*)gC + vb * i, (size_t)vb);                      \
    }                                                                          \
    free(s); free(C);                                                          \
    return 0;                                                                  \
}                                                                              \
                                                                               \
/* Batched key-value merge: segment q merges A[a_off[q] : a_off[q+1]) with     \
 * B[b_off[q] : b_off[q+1]) into C starting at a_off[q] + b_off[q]. */         \
int orc_batched_merge_kv_##SUF(int64_t nseg, const int64_t* a_off,             \
                               const int64_t* b_off,                           \
                               const T* A, const void* Av,                     \
                               const T* B, const void* Bv, int64_t vb,         \
                               T* C, void* Cv)                                 \
{                                                                              \
    for (int64_t q = 0; q < nseg; ++q) {                                       \
        int64_t a0 = a_off[q], m = a_off[q+1] - a_off[q];                      \
        int64_t b0 = b_off[q], n = b_off[q+1] - b_off[q];                      \
        int64_t c0 = a0 + b0;                                                  \
        if (orc_merge_kv_##SUF(A + a0, (const char*)Av + vb * a0, m,           \
                               B + b0, (const char*)Bv + vb * b0, n, vb,       \
                               C + c0, (char*)Cv + vb * c0, 0) != 0)           \
            return -1;                                                         \
    }                                                                          \
    return 0;                                                                  \
}                                                                              \
                                                                               \
int orc_batched_merge_grad_##SUF(int64_t nseg, const int64_t* a_off,           \
                                 const int64_t* b_off,                         \
                                 const T* A, const T* B, const void* gC,       \
                                 int64_t vb, void* gA, void* gB)               \
{                                                                              \
    for (int64_t q = 0; q < nseg; ++q) {                                       \
        int64_t a0 = a_off[q], m = a_off[q+1] - a_off[q];                      \
        int64_t b0 = b_off[q], n = b_off[q+1] - b_off[q];                      \
        int64_t c0 = a0 + b0;                                                  \
        if (orc_merge_grad_##SUF(A + a0, m, B + b0, n,                         \
                                 (const char*)gC + vb * c0, vb,                \
                                 (char*)gA + vb * a0, (char*)gB + vb * b0)     \
            != 0) return -1;                                                   \
    }                                                                          \
    return 0;                                                                  \
}                                                                              \
                                                                               \
/* One pass of a bottom-up merge sort over X[0, N): run pair q holds           \
 * X[2qw, 2qw+w) (the "A" run) and X[2qw+w, min(2qw+2w, N)) (the "B" run);     \
 * the pair is stably merged into Y[2qw, min(2qw+2w, N)).  The payload moves   \
 * with the key; src (nullable) maps every Y position to its X position. */    \
int orc_merge_pass_##SUF(const T* X, const void* Xv, int64_t N, int64_t w,     \
                         int64_t vb, T* Y, void* Yv, int64_t* src)             \
{                                                                              \
    for (int64_t a0 = 0; a0 < N; a0 += 2 * w) {                                \
        int64_t m = orc_min64(w, N - a0);                                      \
        int64_t b0 = a0 + m;                                                   \
        int64_t n = orc_min64(w, N - b0);                                      \
        int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (m + n + 1));          \
        if (!s) return -1;                                                     \
        orc_merge_##SUF(X + a0, m, X + b0, n, Y + a0, s);                      \
        for (int64_t i = 0; i < m + n; ++i) {                                  \
            int64_t from = a0 + s[i];  /* A run then B run are adjacent */     \
            if (vb) memcpy((char*)Yv + vb * (a0 + i),                          \
                           (const char*)Xv + vb * from, (size_t)vb);           \
            if (src) src[a0 + i] = from;                                       \
        }                                                                      \
        free(s);                                                               \
    }                                                                          \
    return 0;                                                                  \
}                                                                              \
                                                                               \
/* Algorithm 2 (Section 3), processing element r of p: output block            \
 * [floor(r(m+n)/p), floor((r+1)(m+n)/p)), both ends co-ranked with            \
 * Algorithm 1, then a sequential stable merge of the two input blocks.        \
 * The products r(m+n) are formed in 64-bit integers. */                       \
typedef struct {                                                               \
    const T* A; int64_t m; const T* B; int64_t n; T* C;                        \
    int64_t r, p; int64_t count; int64_t j0, j1;                               \
} orc_pe_##SUF;                                                                \
                                                                               \
static void* orc_pe_run_##SUF(void* arg)                                       \
{                                                                              \
    orc_pe_##SUF* pe = (orc_pe_##SUF*)arg;                                     \
    int64_t mn = pe->m + pe->n;                                                \
    int64_t i0 = pe->r * mn / pe->p;                                           \
    int64_t i1 = (pe->r + 1) * mn / pe->p;                                     \
    int64_t j0, k0, j1, k1;                                                    \
    orc_co_rank_##SUF(pe->A, pe->m, pe->B, pe->n, i0, &j0, &k0, 0, 0);         \
    orc_co_rank_##SUF(pe->A, pe->m, pe->B, pe->n, i1, &j1, &k1, 0, 0);         \
    orc_merge_##SUF(pe->A + j0, j1 - j0, pe->B + k0, k1 - k0, pe->C + i0, 0);  \
    pe->count = i1 - i0; pe->j0 = j0; pe->j1 = j1;                             \
    return 0;                                                                  \
}                                                                              \
                                                                               \
/* counts (nullable, p entries): elements merged by each processing element. \
 * Returns 0, or -1 if a thread could not be started. */                       \
int orc_parallel_merge_##SUF(const T* A, int64_t m, const T* B, int64_t n,     \
                             T* C, int64_t p, int64_t* counts)                 \
{                                                                              \
    if (p < 1) return -1;                                                      \
    orc_pe_##SUF* pes = (orc_pe_##SUF*)calloc((size_t)p, sizeof(orc_pe_##SUF));\
    pthread_t* th = (pthread_t*)calloc((size_t)p, sizeof(pthread_t));          \
    if (!pes || !th) { free(pes); free(th); return -1; }                       \
    int rc = 0;                                                                \
    int64_t started = 0;                                                       \
    for (int64_t r = 0; r < p; ++r) {                                          \
        pes[r].A = A; pes[r].m = m; pes[r].B = B; pes[r].n = n; pes[r].C = C;  \
        pes[r].r = r; pes[r].p = p;                                            \
        if (r == 0) continue; /* the calling thread is PE 0 */                 \
        if (pthread_create(&th[r], 0, orc_pe_run_##SUF, &pes[r]) != 0) {       \
            rc = -1; break;                                                    \
        }                                                                      \
        started = r;                                                           \
    }                                                                          \
    if (rc == 0) orc_pe_run_##SUF(&pes[0]);                                    \
    for (int64_t r = 1; r <= started; ++r) pthread_join(th[r], 0);             \
    if (rc == 0 && counts)                                                     \
        for (int64_t r = 0; r < p; ++r) counts[r] = pes[r].count;              \
    free(pes); free(th);                                                       \
    return rc;                                                                 \
}

ORC_DEFINE(i32, int32_t)
ORC_DEFINE(u32, uint32_t)
ORC_DEFINE(i64, int64_t)
ORC_DEFINE(u64, uint64_t)
