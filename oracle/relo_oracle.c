/*
 * CPU ORACLE for passive 2-D global relocalization scoring — TEST INFRASTRUCTURE.
 *
 * Plain, slow, FP64/int64 C that restates, step by step, what the paper's
 * scoring path computes: the EDT lookup table (Sec. III-A item 3), the
 * panoramic map-synthesized scan (Eq. 13), SMAD (Eq. 16-20), and TAM
 * (Eq. 23-31); the metrics the paper sets against them: CAER (Eq. 21,
 * Remark 5) in place of SMAD, and the likelihood-field sum (Eq. 32), its
 * normalised form (Eq. 33) and the arithmetic-mean fusion (Eq. 34) in place
 * of TAM; and the ICP refinement of the local top-k poses with their
 * re-evaluation at continuous poses (Sec. III overview, Remark 2).  Only tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library; the GPU library never does.  It shares no code,
 * header or table with the GPU library.
 *
 * Quantisation points (integer semantics shared *by definition* with the GPU
 * path; each side implements them independently):
 *   - occupied cell  <=> value >= 65; unknown (< 0) is free for EDT and rays;
 *   - beam directions D_j = llround((cos, sin)(2 pi j / N_s) * 2^30);
 *   - real ranges R_i = llrint(z_i * 65536 / res) (cells, Q16);
 *   - synthesized range = floor(sqrt(|dcell|^2 * 2^32)) (cells, Q16), 0 = no hit;
 *   - beam endpoint cell = hypothesis cell + round-half-up(R_i * D / 2^46).
 * Every floating-point expression on which an integer decision depends is
 * written the same way on both sides and compiled without FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_E_INVALID (-1)
#define OR_E_BEAM_GRID (-2)
#define OR_E_NO_VALID_BEAMS (-7)

#define TWO_PI (2.0 * M_PI)

static int is_occupied(int8_t v) { return v >= 65; }

static int64_t floor_div_pow2(int64_t a, int sh) {
    /* floor(a / 2^sh) written without relying on >> of negative numbers */
    int64_t d = (int64_t)1 << sh;
    int64_t q = a / d;
    if ((a % d) != 0 && a < 0) q -= 1;
    return q;
}

static int64_t isqrt64(int64_t n) {
    /* floor(sqrt(n)) for 0 <= n < 2^62, exact */
    int64_t r = (int64_t)sqrt((double)n);
    while (r > 0 && r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r;
}

/* ================================================================================
 * EDT lookup table (Sec. III-A item 3): squared distance, in cells, from each cell
 * centre to the nearest occupied cell centre.  d2 = -1 when the map has no
 * occupied cell at all.
 * ============================================================================== */

/* Definition, written out: min over every occupied cell.  O(cells * occupied). */
int64_t oracle_d2_brute(const int8_t *grid, int W, int H, int x, int y) {
    int64_t best = -1;
    for (int oy = 0; oy < H; ++oy)
        for (int ox = 0; ox < W; ++ox)
            if (is_occupied(grid[(size_t)oy * W + ox])) {
                int64_t d2 = (int64_t)(x - ox) * (x - ox) + (int64_t)(y - oy) * (y - oy);
                if (best < 0 || d2 < best) best = d2;
            }
    return best;
}

/*
 * Same minimum, separated by axes: min_{x'} [ (x-x')^2 + g2(x', y) ], where
 * g2(x', y) = min over occupied y' in column x' of (y-y')^2 comes from one
 * downward and one upward sweep per column.  The row minimum visits x' in
 * increasing |x - x'| and stops once (x - x')^2 alone is no smaller than the
 * best sum found, since no further column can then be closer.
 */
void oracle_edt_full(const int8_t *grid, int W, int H, int64_t *d2, int n_threads) {
    int64_t *g2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)W * H);   /* column term, -1 = none */
    (void)n_threads;
#ifdef _OPENMP
    #pragma omp parallel for num_threads(n_threads > 0 ? n_threads : 1) schedule(static)
#endif
    for (int x = 0; x < W; ++x) {
        int64_t last = -1;
        for (int y = 0; y < H; ++y) {
            if (is_occupied(grid[(size_t)y * W + x])) last = y;
            g2[(size_t)y * W + x] = last < 0 ? -1 : (y - last);
        }
        int64_t next = -1;
        for (int y = H - 1; y >= 0; --y) {
            if (is_occupied(grid[(size_t)y * W + x])) next = y;
            int64_t up = g2[(size_t)y * W + x];
            int64_t dn = next < 0 ? -1 : next - y;
            int64_t g = up < 0 ? dn : (dn < 0 ? up : (up < dn ? up : dn));
            g2[(size_t)y * W + x] = g < 0 ? -1 : g * g;
        }
    }
#ifdef _OPENMP
    #pragma omp parallel for num_threads(n_threads > 0 ? n_threads : 1) schedule(static)
#endif
    for (int y = 0; y < H; ++y) {
        const int64_t *row = g2 + (size_t)y * W;
        for (int x = 0; x < W; ++x) {
            int64_t best = row[x];
            for (int64_t dx = 1; dx < W && (best < 0 || dx * dx < best); ++dx) {
                int64_t xs[2] = {x - dx, x + dx};
                for (int k = 0; k < 2; ++k) {
                    if (xs[k] < 0 || xs[k] >= W || row[xs[k]] < 0) continue;
                    int64_t d = dx * dx + row[xs[k]];
                    if (best < 0 || d < best) best = d;
                }
            }
            d2[(size_t)y * W + x] = best;
        }
    }
    free(g2);
}

/*
 * min(d2(x, y), cap) at one cell by an outward search that stops once no
 * unvisited cell can be closer than the best found: column offsets dx are
 * visited in increasing |dx| while dx^2 < best, and within a column rows in
 * increasing |dy| while dx^2 + dy^2 < best.  Returns cap when nothing is
 * closer than cap.
 */
int64_t oracle_d2_capped(const int8_t *grid, int W, int H, int x, int y, int64_t cap) {
    int64_t best = cap;
    for (int64_t dx = 0; dx * dx < best; ++dx) {
        for (int side = 0; side < (dx == 0 ? 1 : 2); ++side) {
            int64_t cx = side ? x - dx : x + dx;
            if (cx < 0 || cx >= W) continue;
            for (int64_t dy = 0; dx * dx + dy * dy < best; ++dy) {
                int64_t r1 = y + dy, r2 = y - dy;
                int hit = (r1 < H && is_occupied(grid[(size_t)r1 * W + cx])) ||
                          (dy > 0 && r2 >= 0 && is_occupied(grid[(size_t)r2 * W + cx]));
                if (hit) { best = dx * dx + dy * dy; break; }
                if (r1 >= H - 1 && r2 <= 0) break;
            }
        }
    }
    return best;
}

/* ================================================================================
 * Sensor plan: beam grid (Eq. 11, 14), FoV intervals (Eq. 12), directions.
 * ============================================================================== */

/*
 * From the beam angles, find N_s (Eq. 14: 2 pi over the angular step) and the
 * panoramic index b_i of every beam.  Consecutive angles (unwrapped, so a
 * scan may cross +-pi) differ by a whole number of steps, one step for a
 * contiguous FoV and more across an occluded sector (Eq. 12); that number is
 * the difference over the smallest difference, rounded, and the step is the
 * span over the total.  Every angle must sit within 1e-3 steps of a multiple
 * of 2 pi / N_s, and no two beams may share an index.
 */
int oracle_beam_grid(const float *ang, int n, int32_t *ns_out, int32_t *b_out) {
    if (n < 2) return OR_E_BEAM_GRID;
    /* unwrapped consecutive differences; the smallest is about one grid step */
    double *dif = (double *)malloc(sizeof(double) * (size_t)(n - 1));
    double dmin = INFINITY, span = 0.0;
    for (int i = 1; i < n; ++i) {
        double d = (double)ang[i] - (double)ang[i - 1];
        if (d < 0.0) d += TWO_PI;
        dif[i - 1] = d;
        span += d;
        if (d < dmin) dmin = d;
    }
    if (!(dmin > 0.0)) { free(dif); return OR_E_BEAM_GRID; }
    /* whole grid steps between consecutive beams, then step = span / steps */
    long long steps = 0;
    for (int i = 0; i < n - 1; ++i) steps += llround(dif[i] / dmin);
    free(dif);
    double step = span / (double)steps;
    long long ns = llround(TWO_PI / step);
    if (ns < n || ns > 65536) return OR_E_BEAM_GRID;
    double dphi = TWO_PI / (double)ns;
    char *seen = (char *)calloc((size_t)ns, 1);
    for (int i = 0; i < n; ++i) {
        double q = (double)ang[i] / dphi;
        long long k = llround(q);
        if (fabs(q - (double)k) > 1e-3) { free(seen); return OR_E_BEAM_GRID; }
        long long b = ((k % ns) + ns) % ns;
        if (seen[b]) { free(seen); return OR_E_BEAM_GRID; }
        seen[b] = 1;
        b_out[i] = (int32_t)b;
    }
    free(seen);
    *ns_out = (int32_t)ns;
    return OR_OK;
}

/* D_j = llround((cos, sin)(2 pi j / N_s) * 2^30), j in [0, N_s) */
void oracle_directions(int ns, int64_t *D) {
    for (int j = 0; j < ns; ++j) {
        double a = TWO_PI * (double)j / (double)ns;
        D[2 * j] = llround(ldexp(cos(a), 30));
        D[2 * j + 1] = llround(ldexp(sin(a), 30));
    }
}

/*
 * FoV intervals (Eq. 12): the panoramic indices covered by the sensor's beams,
 * as maximal cyclic runs [u_k, u_k + len_k - 1].  Returns K.
 */
int oracle_intervals(const int32_t *b, int n, int ns, int32_t *u_out, int32_t *len_out) {
    char *cov = (char *)calloc((size_t)ns, 1);
    for (int i = 0; i < n; ++i) cov[b[i]] = 1;
    int K = 0;
    if (n == ns) { u_out[0] = 0; len_out[0] = ns; free(cov); return 1; }
    for (int j = 0; j < ns; ++j) {
        int prev = (j + ns - 1) % ns;
        if (cov[j] && !cov[prev]) {
            int len = 0;
            while (cov[(j + len) % ns] && len < ns) ++len;
            u_out[K] = j;
            len_out[K] = len;
            ++K;
        }
    }
    free(cov);
    return K;
}

/* R_i = llrint(z_i * 65536 / res) for valid beams (finite, 0 < z < max_range), else 0 */
void oracle_ranges_q16(const float *z, int n, float max_range, double res, int64_t *R, uint8_t *valid) {
    for (int i = 0; i < n; ++i) {
        float v = z[i];
        int ok = isfinite(v) && v > 0.0f && v < max_range;
        valid[i] = (uint8_t)ok;
        R[i] = ok ? llrint((double)v * 65536.0 / res) : 0;
    }
}

/* ================================================================================
 * Panoramic map-synthesized scan (Eq. 13) by integer ray casting.
 * ============================================================================== */

/*
 * Casts one ray from the centre of cell (hx, hy) along D = (Dx, Dy) (Q30).
 * Cells are entered in the order of the ray's boundary crossings: the k-th
 * x-boundary (k = 0, 1, ...) is crossed at parameter (2k+1)/(2|Dx|) and the
 * l-th y-boundary at (2l+1)/(2|Dy|); x is stepped when (2k+1)|Dy| <= (2l+1)|Dx|
 * (an exact tie at a cell corner steps x first).  The ray stops with no hit on
 * leaving the map or on entering a cell whose centre lies beyond the maximum
 * range ((dx^2 + dy^2) * 2^32 > rmax_q16^2), and with a hit on entering an
 * occupied cell.  Returns floor(sqrt((dx^2 + dy^2) * 2^32)) for a hit, else 0.
 */
int64_t oracle_cast_ray(const int8_t *grid, int W, int H, int hx, int hy, int64_t Dx, int64_t Dy,
                        int64_t rmax_q16, int32_t *hit_x, int32_t *hit_y, int64_t *steps) {
    int64_t ax = Dx < 0 ? -Dx : Dx, ay = Dy < 0 ? -Dy : Dy;
    int sx = Dx > 0 ? 1 : -1, sy = Dy > 0 ? 1 : -1;
    int64_t k = 0, l = 0;
    int64_t cx = hx, cy = hy;
    int64_t n = 0;
    int64_t r2max = rmax_q16 * rmax_q16;
    for (;;) {
        if ((2 * k + 1) * ay <= (2 * l + 1) * ax) { cx += sx; ++k; }
        else { cy += sy; ++l; }
        ++n;
        if (cx < 0 || cy < 0 || cx >= W || cy >= H) break;
        int64_t dx = cx - hx, dy = cy - hy;
        int64_t c2 = dx * dx + dy * dy;
        if (c2 * ((int64_t)1 << 32) > r2max) break;
        if (is_occupied(grid[(size_t)cy * W + cx])) {
            if (hit_x) *hit_x = (int32_t)cx;
            if (hit_y) *hit_y = (int32_t)cy;
            if (steps) *steps = n;
            return isqrt64(c2 << 32);
        }
    }
    if (hit_x) *hit_x = -1;
    if (hit_y) *hit_y = -1;
    if (steps) *steps = n;
    return 0;
}

/* all N_s synthesized ranges of one hypothesis; hit cells optional */
void oracle_synth_scan(const int8_t *grid, int W, int H, int hx, int hy, int ns, const int64_t *D,
                       int64_t rmax_q16, int64_t *ranges, int32_t *hit_x, int32_t *hit_y) {
    for (int j = 0; j < ns; ++j)
        ranges[j] = oracle_cast_ray(grid, W, H, hx, hy, D[2 * j], D[2 * j + 1], rmax_q16,
                                    hit_x ? &hit_x[j] : NULL, hit_y ? &hit_y[j] : NULL, NULL);
}

/* ================================================================================
 * SMAD (Eq. 16-20), in the direct (no prefix sum) form.
 * ============================================================================== */

/*
 * For every hypothesis: SMAD numerator
 *     |sum_real - W_m|,  W_m = sum_k sum_{t < len_k} syn[(u_k + t + m) mod N_s],
 * where sum_real is the sum of the real Q16 ranges (invalid beams = 0).  Both
 * means of Eq. 16 and Eq. 18 share the denominator sum_k |I_k|, so comparing
 * numerators compares SMAD.  Eq. 20: m = 0 only when lambda >= 0.9, else the
 * minimum over m in {0, n_enum, 2 n_enum, ...} (ties keep the smaller m).
 * Outputs the numerator and the minimising m per hypothesis.
 */
void oracle_smad(const int8_t *grid, int W, int H, const int32_t *hyp_xy, int n_hyp, int ns,
                 const int64_t *D, int64_t rmax_q16, const int32_t *u, const int32_t *len, int K,
                 int64_t sum_real, int n_enum, int panoramic, int64_t *num_out, int32_t *m_out,
                 int n_threads) {
    (void)n_threads;
#ifdef _OPENMP
    #pragma omp parallel for num_threads(n_threads > 0 ? n_threads : 1) schedule(dynamic, 4)
#endif
    for (int h = 0; h < n_hyp; ++h) {
        int64_t *syn = (int64_t *)malloc(sizeof(int64_t) * ns);
        oracle_synth_scan(grid, W, H, hyp_xy[2 * h], hyp_xy[2 * h + 1], ns, D, rmax_q16, syn, NULL, NULL);
        int64_t best = -1;
        int32_t best_m = 0;
        int m_end = panoramic ? 1 : ns;
        for (int m = 0; m < m_end; m += n_enum) {
            int64_t Wm = 0;
            for (int k = 0; k < K; ++k)
                for (int t = 0; t < len[k]; ++t) Wm += syn[(u[k] + t + m) % ns];
            int64_t d = sum_real - Wm;
            if (d < 0) d = -d;
            if (best < 0 || d < best) { best = d; best_m = m; }
        }
        num_out[h] = best;
        m_out[h] = best_m;
        free(syn);
    }
}

/*
 * CAER (Eq. 21) for every hypothesis: the numerator
 *     sum_i |R_i - syn[(b_i + m) mod N_s]|
 * over every beam i of the FoV intervals (the intervals are exactly the
 * beams' panoramic indices b_i; an invalid beam carries the placeholder 0, as
 * in SMAD), minimised over the same orientations as SMAD (Eq. 20: m = 0 only
 * when lambda >= 0.9); the denominator sum_k |I_k| is shared by every
 * hypothesis and orientation, so numerators compare CAER.  Ties keep the
 * smaller m.  R holds the n beams' Q16 ranges (0 for invalid ones).
 */
void oracle_caer(const int8_t *grid, int W, int H, const int32_t *hyp_xy, int n_hyp, int ns,
                 const int64_t *D, int64_t rmax_q16, const int32_t *b, const int64_t *R, int n, int n_enum,
                 int panoramic, int64_t *num_out, int32_t *m_out, int n_threads) {
    (void)n_threads;
#ifdef _OPENMP
    #pragma omp parallel for num_threads(n_threads > 0 ? n_threads : 1) schedule(dynamic, 4)
#endif
    for (int h = 0; h < n_hyp; ++h) {
        int64_t *syn = (int64_t *)malloc(sizeof(int64_t) * ns);
        oracle_synth_scan(grid, W, H, hyp_xy[2 * h], hyp_xy[2 * h + 1], ns, D, rmax_q16, syn, NULL, NULL);
        int64_t best = -1;
        int32_t best_m = 0;
        int m_end = panoramic ? 1 : ns;
        for (int m = 0; m < m_end; m += n_enum) {
            int64_t e = 0;
            for (int i = 0; i < n; ++i) {
                int64_t d = R[i] - syn[(b[i] + m) % ns];
                e += d < 0 ? -d : d;
            }
            if (best < 0 || e < best) { best = e; best_m = m; }
        }
        num_out[h] = best;
        m_out[h] = best_m;
        free(syn);
    }
}

/* ================================================================================
 * TAM (Eq. 23-31) for a list of (hypothesis, m) pairs.
 * ============================================================================== */

typedef struct {
    double z_hit, sigma_hit, z_rand, eps;
    double res, d_max;
    double a_mid, a_low;       /* Eq. 25 retention ratios (already evaluated at lambda) */
    int metric;                /* 0 TAM (Eq. 31), 1 TAM_mean (Eq. 34), 2 wp_baseline (Eq. 33), 3 wp_LF (Eq. 32) */
} tam_params;

static int cmp_desc(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/*
 * The score of Eq. 23-31 (or of the metric p->metric selects, see tam_one)
 * from the N beam-endpoint obstacle distances dist[0 .. N) (metres); ell is
 * scratch of N doubles.  NaN when N = 0.
 */
static double score_of_distances(const double *dist, double *ell, int N, const tam_params *p, double *comp) {
    if (N == 0) return NAN;
    for (int i = 0; i < N; ++i) {
        double d = dist[i];
        ell[i] = log(p->z_hit * exp(-(d * d) / (2.0 * p->sigma_hit * p->sigma_hit)) + p->z_rand + p->eps);
    }
    qsort(ell, (size_t)N, sizeof(double), cmp_desc);
    int kf = N;
    int km = (int)floor(p->a_mid * (double)N); if (km < 1) km = 1;
    int kl = (int)floor(p->a_low * (double)N); if (kl < 1) kl = 1;
    int ks[3] = {kf, km, kl};
    double mean[3];
    for (int t = 0; t < 3; ++t) {
        double s = 0.0;
        for (int i = 0; i < ks[t]; ++i) s += ell[i];
        mean[t] = s / ks[t];
    }
    /* median of three */
    double lf = 0.0;   /* Eq. 32: every beam, before any retention */
    for (int i = 0; i < N; ++i) lf += ell[i];
    double a = mean[0], bb = mean[1], c3 = mean[2], med;
    if ((a <= bb && bb <= c3) || (c3 <= bb && bb <= a)) med = bb;
    else if ((bb <= a && a <= c3) || (c3 <= a && a <= bb)) med = a;
    else med = c3;
    double wp = exp(med);
    double dmean = 0.0;
    for (int i = 0; i < N; ++i) dmean += dist[i];
    dmean /= N;
    double var = 0.0;
    for (int i = 0; i < N; ++i) var += (dist[i] - dmean) * (dist[i] - dmean);
    var /= N;
    double dmin = p->res / 2.0;
    double dt = dmean < dmin ? dmin : dmean;
    if (dt > p->d_max) dt = p->d_max;
    double sd = 1.0 - (dt - dmin) / (p->d_max - dmin);
    double c = exp(-0.5 * var);
    double T;
    switch (p->metric) {
    case 1: T = (wp + sd + c) / 3.0; break;          /* Eq. 34 */
    case 2: T = sqrt(exp(lf / N) * sd); break;        /* Eq. 33 */
    case 3: T = lf; break;                            /* Eq. 32 */
    default: T = cbrt(wp * sd * c); break;            /* Eq. 31 */
    }
    if (comp) { comp[0] = med; comp[1] = wp; comp[2] = sd; comp[3] = c; comp[4] = dmean; }
    return T;
}

/*
 * One TAM score.  For each valid beam i at orientation m the endpoint cell is
 * the hypothesis cell plus round-half-up(R_i * D_{(b_i + m) mod N_s} / 2^46);
 * its obstacle distance is d_i = res * sqrt(min(d2, C)), C = (d_max/res)^2,
 * and an endpoint off the map takes d_max.  Then (Eq. 23) l_i, (Eq. 24) the
 * descending sort, (Eq. 26) k_full = N, k_mid = max(1, floor(a_mid N)),
 * k_low = max(1, floor(a_low N)), (Eq. 27) the median of the three top-k
 * means, (Eq. 28) exp of it, (Eq. 29) s_d with d_min = res / 2, (Eq. 30) c from
 * the population variance of the d_i, and (Eq. 31) the cube root of the
 * product.  comp[0..4] (optional) receives L_bar, wp, s_d, c, mean d.
 * With p->metric the score is instead the arithmetic mean (wp + s_d + c) / 3
 * of the same components (Eq. 34), the likelihood-field sum
 * wp_LF = sum of l_i over all N beams (Eq. 32), or its normalised form
 * (exp(wp_LF / N) s_d)^(1/2) (Eq. 33: no retention, no c).
 */
static double tam_one(const int8_t *grid, const int64_t *d2tab, int W, int H, int hx, int hy, int m, int ns,
                      const int64_t *D, const int32_t *b, const int64_t *R, const uint8_t *valid, int n,
                      const tam_params *p, double *dist, double *ell, double *comp) {
    int64_t C = llround(p->d_max / p->res);
    C = C * C;
    int N = 0;
    for (int i = 0; i < n; ++i) {
        if (!valid[i]) continue;
        int j = (b[i] + m) % ns;
        int64_t ox = floor_div_pow2(R[i] * D[2 * j] + ((int64_t)1 << 45), 46);
        int64_t oy = floor_div_pow2(R[i] * D[2 * j + 1] + ((int64_t)1 << 45), 46);
        int64_t ex = hx + ox, ey = hy + oy;
        int64_t q;
        if (ex < 0 || ey < 0 || ex >= W || ey >= H) q = C;
        else if (d2tab) {
            q = d2tab[(size_t)ey * W + ex];
            if (q < 0 || q > C) q = C;
        } else q = oracle_d2_capped(grid, W, H, (int)ex, (int)ey, C);
        dist[N] = p->res * sqrt((double)q);
        ++N;
    }
    return score_of_distances(dist, ell, N, p, comp);
}

/*
 * TAM scores for n_pairs (hypothesis cell, m) pairs.  d2tab (row-major, from
 * oracle_edt_full) may be NULL, in which case distances come from
 * oracle_d2_capped.  params: z_hit, sigma_hit, z_rand, eps, res, d_max, a_mid,
 * a_low, metric (0-3, see tam_one).  comp (optional) receives 5 components per
 * pair.
 */
void oracle_tam(const int8_t *grid, const int64_t *d2tab, int W, int H, const int32_t *pair_xy,
                const int32_t *pair_m, int n_pairs, int ns, const int64_t *D, const int32_t *b,
                const int64_t *R, const uint8_t *valid, int n, const double *params, double *T_out,
                double *comp, int n_threads) {
    tam_params p = {params[0], params[1], params[2], params[3], params[4], params[5], params[6], params[7],
                    (int)params[8]};
    (void)n_threads;
#ifdef _OPENMP
    #pragma omp parallel for num_threads(n_threads > 0 ? n_threads : 1) schedule(dynamic, 8)
#endif
    for (int q = 0; q < n_pairs; ++q) {
        double *dist = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
        double *ell = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
        T_out[q] = tam_one(grid, d2tab, W, H, pair_xy[2 * q], pair_xy[2 * q + 1], pair_m[q], ns, D, b, R,
                           valid, n, &p, dist, ell, comp ? &comp[5 * q] : NULL);
        free(dist);
        free(ell);
    }
}

/* ================================================================================
 * ICP refinement and re-evaluation at continuous poses: the framework's last
 * step (Sec. III overview: the local top-k poses are aligned to the whole map
 * by ICP, then scored again; Remark 2 names the operator).  The paper does not
 * specify the ICP variant; this is point-to-point ICP against the centres of
 * occupied cells, pairs found through the exact EDT and kept within d_max.
 * ============================================================================== */

/*
 * The nearest occupied cell to cell (x, y) when its squared distance d2 (the
 * exact EDT value there) is at most cap: the cells (x + dx, y + dy) with
 * dx^2 + dy^2 = d2 are tried in order of increasing dy, then increasing dx,
 * and the first occupied one on the map is returned (1, with *ox, *oy); 0 when
 * (x, y) is off the map, no cell is occupied, or d2 > cap.
 */
int oracle_nearest_occupied(const int8_t *grid, const int64_t *d2tab, int W, int H, int x, int y, int64_t cap,
                            int *ox, int *oy) {
    if (x < 0 || y < 0 || x >= W || y >= H) return 0;
    int64_t d2 = d2tab ? d2tab[(size_t)y * W + x] : oracle_d2_capped(grid, W, H, x, y, cap + 1);
    if (d2 < 0 || d2 > cap) return 0;
    int64_t r = isqrt64(d2);
    for (int64_t dy = -r; dy <= r; ++dy) {
        int64_t rest = d2 - dy * dy;
        int64_t s = isqrt64(rest);
        if (s * s != rest) continue;
        for (int sign = -1; sign <= 1; sign += 2) {
            int64_t dx = sign * s;
            if (sign > 0 && s == 0) break;   /* dx = 0 was tried as -0 */
            int64_t cx = x + dx, cy = y + dy;
            if (cx < 0 || cy < 0 || cx >= W || cy >= H) continue;
            if (is_occupied(grid[(size_t)cy * W + cx])) { *ox = (int)cx; *oy = (int)cy; return 1; }
        }
    }
    return 0;
}

/*
 * The rigid motion (rotation phi, translation t) that minimises
 * sum_i |R(phi) w_i + t - c_i|^2 over n point pairs (w, c interleaved x, y):
 * with the centroids mw, mc and the centred points w', c',
 * phi = atan2(sum (w'_x c'_y - w'_y c'_x), sum (w'_x c'_x + w'_y c'_y)) and
 * t = mc - R(phi) mw.  Returns 0 when n < 2.
 */
int oracle_rigid_fit(const double *w, const double *c, int n, double *phi, double *tx, double *ty) {
    if (n < 2) return 0;
    double mwx = 0, mwy = 0, mcx = 0, mcy = 0;
    for (int i = 0; i < n; ++i) { mwx += w[2 * i]; mwy += w[2 * i + 1]; mcx += c[2 * i]; mcy += c[2 * i + 1]; }
    mwx /= n; mwy /= n; mcx /= n; mcy /= n;
    double sxy = 0, sdot = 0;
    for (int i = 0; i < n; ++i) {
        double ax = w[2 * i] - mwx, ay = w[2 * i + 1] - mwy, bx = c[2 * i] - mcx, by = c[2 * i + 1] - mcy;
        sxy += ax * by - ay * bx;
        sdot += ax * bx + ay * by;
    }
    double f = atan2(sxy, sdot);
    *phi = f;
    *tx = mcx - (cos(f) * mwx - sin(f) * mwy);
    *ty = mcy - (sin(f) * mwx + cos(f) * mwy);
    return 1;
}

/*
 * A beam's world point at pose (x, y, theta): the point at range z along the
 * world direction theta + a, w = (x + z cos(theta + a), y + z sin(theta + a)),
 * and the cell that contains it, (floor(w_x / res), floor(w_y / res)).
 */
static void world_point(double x, double y, double theta, double z, double a, double res, double *wx, double *wy,
                        int *cx, int *cy) {
    *wx = x + z * cos(theta + a);
    *wy = y + z * sin(theta + a);
    *cx = (int)floor(*wx / res);
    *cy = (int)floor(*wy / res);
}

/*
 * ICP from pose = (x, y, theta) (metres, radians; refined in place) for n
 * beams with sensor-frame ranges z (metres) and angles a.  Each iteration maps
 * beam i to its world point (world_point), pairs it with the centre of the
 * nearest occupied cell to the cell it falls in (kept when that squared cell
 * distance is at most C, i.e. within d_max), fits the rigid motion of the
 * pairs and composes it with the pose.  It stops after iters iterations, when
 * fewer than 2 pairs remain, or when the motion is below 1e-9 rad and 1e-9 m.
 * Returns the iterations applied.
 */
int oracle_icp(const int8_t *grid, const int64_t *d2tab, int W, int H, double res, int64_t C, const double *z,
               const double *a, int n, int iters, double *pose) {
    double *w = (double *)malloc(sizeof(double) * 2 * (n > 0 ? n : 1));
    double *c = (double *)malloc(sizeof(double) * 2 * (n > 0 ? n : 1));
    int it = 0;
    for (; it < iters; ++it) {
        int k = 0;
        for (int i = 0; i < n; ++i) {
            double wx, wy;
            int cx, cy, ox, oy;
            world_point(pose[0], pose[1], pose[2], z[i], a[i], res, &wx, &wy, &cx, &cy);
            if (!oracle_nearest_occupied(grid, d2tab, W, H, cx, cy, C, &ox, &oy)) continue;
            w[2 * k] = wx; w[2 * k + 1] = wy;
            c[2 * k] = (ox + 0.5) * res; c[2 * k + 1] = (oy + 0.5) * res;
            ++k;
        }
        double f, tx, ty;
        if (!oracle_rigid_fit(w, c, k, &f, &tx, &ty)) break;
        double nx = cos(f) * pose[0] - sin(f) * pose[1] + tx;
        double ny = sin(f) * pose[0] + cos(f) * pose[1] + ty;
        double moved = fabs(nx - pose[0]) + fabs(ny - pose[1]);
        pose[0] = nx; pose[1] = ny; pose[2] += f;
        if (fabs(f) < 1e-9 && moved < 1e-9) { ++it; break; }
    }
    free(w);
    free(c);
    return it;
}

/*
 * The score (TAM or the metric params[8] selects) at continuous poses
 * (x, y, theta interleaved) for n beams with sensor-frame ranges z (metres)
 * and angles a: beam i ends in the cell of its world point (world_point); its
 * distance is res * sqrt(min(d2, C)), d_max off the map, as in tam_one.
 * params as oracle_tam.
 */
void oracle_tam_pose(const int8_t *grid, const int64_t *d2tab, int W, int H, const double *poses, int n_poses,
                     const double *z, const double *a, int n, const double *params, double *T_out, int n_threads) {
    tam_params p = {params[0], params[1], params[2], params[3], params[4], params[5], params[6], params[7],
                    (int)params[8]};
    int64_t C = llround(p.d_max / p.res);
    C = C * C;
    (void)n_threads;
#ifdef _OPENMP
    #pragma omp parallel for num_threads(n_threads > 0 ? n_threads : 1) schedule(dynamic, 8)
#endif
    for (int q = 0; q < n_poses; ++q) {
        double *dist = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
        double *ell = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
        const double *ps = poses + 3 * q;
        for (int i = 0; i < n; ++i) {
            double wx, wy;
            int cx, cy;
            world_point(ps[0], ps[1], ps[2], z[i], a[i], p.res, &wx, &wy, &cx, &cy);
            int64_t ex = cx, ey = cy;
            int64_t d2;
            if (ex < 0 || ey < 0 || ex >= W || ey >= H) d2 = C;
            else if (d2tab) {
                d2 = d2tab[(size_t)ey * W + ex];
                if (d2 < 0 || d2 > C) d2 = C;
            } else d2 = oracle_d2_capped(grid, W, H, (int)ex, (int)ey, C);
            dist[i] = p.res * sqrt((double)d2);
        }
        T_out[q] = score_of_distances(dist, ell, n, &p, NULL);
        free(dist);
        free(ell);
    }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
