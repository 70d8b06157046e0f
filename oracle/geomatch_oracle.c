/*
 * geomatch_oracle.c -- plain FP64 CPU oracle for geometry-aware pairwise feature matching
 * (Shah, Deshpande, Narayanan, "Multistage SFM: A Coarse-to-Fine Approach for 3D Reconstruction",
 * arXiv 1512.06235, Sec. 6.2 and Appendix A).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this file: only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark use it.  It shares no code,
 * header or constant with the CUDA library; the two agree only because both follow the paper.
 *
 * What it computes, per image pair (A, B, F, d, ratio p/q), for every query feature i of A in index order:
 *   1. the epipolar line l = F * (x_i, y_i, 1)^T in image B (Sec. 6.2, the line l_q = F_qc p_q; F is an input
 *      with the convention that l lives in image B -- Eq. 1 as printed is the transposed form);
 *   2. the candidate set C_i = { j in B : dist(p'_j, l) <= d }   (Eq. 2, inclusive), with the point-to-line
 *      distance of Eq. 3 read with an absolute value and evaluated as |a x' + b y' + c| <= d * sqrt(a^2+b^2)
 *      (the division is avoided); C_i is found by linear search over all of B (Sec. 6.2.1, "Linear search");
 *   3. the exact squared L2 distance D(i,j) = sum_k (A_ik - B_jk)^2 over the 128-byte descriptors for j in C_i;
 *   4. the two nearest neighbours (Sec. 6.2.2 top-two retrieval; Appendix A Step 4 minimum and next minimum):
 *      (D1, j1) = lexicographic minimum of (D, j), D2 = minimum of D over C_i without j1;
 *   5. Lowe's ratio test (Sec. 2.3): accept j1 iff |C_i| >= 2 and dist1/dist2 < p/q, i.e. in integers
 *      q^2 * D1 < p^2 * D2 (strict, so a tie D1 == D2 rejects).
 *
 * Readings taken where the paper is silent (each is also listed in the design notes):
 *   - floating point: every step of the band test is FP64, round to nearest, left-to-right sums, and this file
 *     must be compiled with -ffp-contract=off so that no multiply-add is fused;
 *   - a line with a == b == 0 has no defined distance: C_i is empty for finite d;
 *   - d == +infinity makes C_i all of B (the band covers the image: exhaustive matching);
 *   - |C_i| < 2 gives no match (the ratio is undefined with one neighbour).
 *
 * Parity pins (tests, CPU): exhaustive matching at d = inf against an independent brute force and
 * scipy's cdist; band membership against exact rational arithmetic and the closed form of a rectified pair;
 * recall of known correspondences on synthetic scenes; the transpose symmetry of the band.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GMO_DIM 128

/* Epipolar line of query point (x, y) in image B: l = F (x, y, 1)^T  (Sec. 6.2, l_q = F_qc p_q).
 * F is row-major.  FP64, left-to-right, no fused multiply-add. */
void gmo_line(const float F[9], float xf, float yf, double out[3])
{
    const double x = (double)xf, y = (double)yf;
    out[0] = ((double)F[0] * x + (double)F[1] * y) + (double)F[2];
    out[1] = ((double)F[3] * x + (double)F[4] * y) + (double)F[5];
    out[2] = ((double)F[6] * x + (double)F[7] * y) + (double)F[8];
}

/* Band membership of point (x', y') for line l (Eqs. 2-3): |a x' + b y' + c| <= d * sqrt(a^2 + b^2).
 * Returns 1 if inside (inclusive), 0 otherwise. */
int gmo_in_band(const double l[3], float d, float xpf, float ypf)
{
    if (isinf(d)) return 1;
    const double a = l[0], b = l[1], c = l[2];
    const double n = sqrt(a * a + b * b);
    if (n == 0.0) return 0;
    const double thr = (double)d * n;
    const double s = (a * (double)xpf + b * (double)ypf) + c;
    return fabs(s) <= thr;
}

/* Exact squared L2 distance of two 128-byte descriptors (Sec. 2.3, L2 norm between descriptors). */
int32_t gmo_dist2(const uint8_t *u, const uint8_t *v)
{
    int32_t acc = 0;
    for (int k = 0; k < GMO_DIM; ++k) {
        const int32_t t = (int32_t)u[k] - (int32_t)v[k];
        acc += t * t;
    }
    return acc;
}

/* Candidate set C_i of one query (Eq. 2 by linear search, Sec. 6.2.1).  Writes the B indices in ascending
 * order to out (capacity cap) and returns |C_i| (which may exceed cap; only cap entries are written). */
int64_t gmo_band_set(const float F[9], float d, float xq, float yq,
                     int32_t nB, const float *xyB, int32_t *out, int64_t cap)
{
    double l[3];
    gmo_line(F, xq, yq, l);
    int64_t cnt = 0;
    for (int32_t j = 0; j < nB; ++j) {
        if (gmo_in_band(l, d, xyB[2 * j], xyB[2 * j + 1])) {
            if (cnt < cap) out[cnt] = j;
            ++cnt;
        }
    }
    return cnt;
}

/* Match one pair (Sec. 6.2 with Appendix A Steps 3-4 semantics).
 * match_j[i] = j1 (index into B) for accepted queries, -1 otherwise.
 * Optional outputs (may be NULL): n_cand = sum_i |C_i| (the exact candidate comparisons),
 * d1/d2 per query (INT32_MAX where undefined).  Returns the number of matches, or -1 on bad arguments. */
int64_t gmo_match_pair(int32_t nA, const float *xyA, const uint8_t *descA,
                       int32_t nB, const float *xyB, const uint8_t *descB,
                       const float F[9], float d, int32_t p, int32_t q,
                       int32_t *match_j, int64_t *n_cand, int32_t *d1_out, int32_t *d2_out)
{
    if (nA < 0 || nB < 0 || q <= 0 || p < 0 || !(d >= 0.0f)) return -1;
    const int64_t p2 = (int64_t)p * p, q2 = (int64_t)q * q;
    int64_t total = 0, matches = 0;
    for (int32_t i = 0; i < nA; ++i) {
        double l[3];
        gmo_line(F, xyA[2 * i], xyA[2 * i + 1], l);
        int32_t D1 = INT32_MAX, D2 = INT32_MAX, j1 = -1;
        int64_t cnt = 0;
        for (int32_t j = 0; j < nB; ++j) {             /* ascending j: ties keep the lowest index */
            if (!gmo_in_band(l, d, xyB[2 * j], xyB[2 * j + 1])) continue;
            ++cnt;
            const int32_t D = gmo_dist2(descA + (size_t)i * GMO_DIM, descB + (size_t)j * GMO_DIM);
            if (D < D1) { D2 = D1; D1 = D; j1 = j; }
            else if (D < D2) { D2 = D; }
        }
        total += cnt;
        int32_t m = -1;
        if (cnt >= 2 && q2 * (int64_t)D1 < p2 * (int64_t)D2) m = j1;
        match_j[i] = m;
        if (m >= 0) ++matches;
        if (d1_out) d1_out[i] = D1;
        if (d2_out) d2_out[i] = D2;
    }
    if (n_cand) *n_cand = total;
    return matches;
}

/* ---- batch over pairs, multithreaded (pairs are independent, Sec. 6.2.3 "Easy parallelization") ---- */

typedef struct {
    int32_t n_images;
    const int32_t *img_n;            /* [n_images] */
    const float *const *img_xy;      /* [n_images] -> n*2 */
    const uint8_t *const *img_desc;  /* [n_images] -> n*128 */
    int32_t n_pairs;
    const int32_t *pair_ab;          /* [n_pairs*2] */
    const float *pair_F;             /* [n_pairs*9] */
    const float *pair_d;             /* [n_pairs] */
    const int32_t *pair_pq;          /* [n_pairs*2] */
    const int64_t *out_off;          /* [n_pairs] offset of each pair's match_j block (n_A entries) */
    int32_t *match_j;
    int64_t *n_cand;                 /* [n_pairs] */
    int64_t next;                    /* shared work counter */
    pthread_mutex_t lock;
    int status;
} gmo_batch;

static void *gmo_worker(void *arg)
{
    gmo_batch *bt = (gmo_batch *)arg;
    for (;;) {
        pthread_mutex_lock(&bt->lock);
        const int64_t k = bt->next++;
        pthread_mutex_unlock(&bt->lock);
        if (k >= bt->n_pairs) break;
        const int32_t a = bt->pair_ab[2 * k], b = bt->pair_ab[2 * k + 1];
        if (a < 0 || b < 0 || a >= bt->n_images || b >= bt->n_images) { bt->status = -1; continue; }
        const int64_t r = gmo_match_pair(bt->img_n[a], bt->img_xy[a], bt->img_desc[a],
                                         bt->img_n[b], bt->img_xy[b], bt->img_desc[b],
                                         bt->pair_F + 9 * k, bt->pair_d[k],
                                         bt->pair_pq[2 * k], bt->pair_pq[2 * k + 1],
                                         bt->match_j + bt->out_off[k], bt->n_cand + k, NULL, NULL);
        if (r < 0) bt->status = -1;
    }
    return NULL;
}

/* Runs gmo_match_pair over all pairs on n_threads host threads.  Returns 0, or -1 on bad arguments. */
int gmo_match_batch(int32_t n_images, const int32_t *img_n, const float *const *img_xy,
                    const uint8_t *const *img_desc, int32_t n_pairs, const int32_t *pair_ab,
                    const float *pair_F, const float *pair_d, const int32_t *pair_pq,
                    const int64_t *out_off, int32_t *match_j, int64_t *n_cand, int32_t n_threads)
{
    gmo_batch bt;
    bt.n_images = n_images; bt.img_n = img_n; bt.img_xy = img_xy; bt.img_desc = img_desc;
    bt.n_pairs = n_pairs; bt.pair_ab = pair_ab; bt.pair_F = pair_F; bt.pair_d = pair_d;
    bt.pair_pq = pair_pq; bt.out_off = out_off; bt.match_j = match_j; bt.n_cand = n_cand;
    bt.next = 0; bt.status = 0;
    pthread_mutex_init(&bt.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 1; t < n_threads; ++t)
        if (pthread_create(&th[started], NULL, gmo_worker, &bt) == 0) ++started;
    gmo_worker(&bt);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&bt.lock);
    return bt.status;
}
