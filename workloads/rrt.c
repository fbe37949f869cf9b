/*
 * Traversability-constrained RRT hypothesis sampler (Sec. III-A, Algorithm 1).
 *
 * This is the seeded generator of positional hypotheses (Eq. 6) that both the
 * CPU oracle and the GPU path consume.  It is input generation, not part of the
 * scoring path, and shares no code with either side.
 *
 * Readings of the paper's helper functions (Sec. III-A items 1-7):
 *   - MinDistToObstacle d_obs(p): a lookup table of per-cell clearance
 *     (distance from the cell centre to the nearest occupied or unknown cell
 *     centre) read at the cell that contains p, as the paper does with its
 *     precomputed table.  The caller supplies the table.
 *   - AdaptiveExpandDist: eta = eta_max if d >= 2r; eta = r if d <= r;
 *     linear between (d=r, eta=r) and (d=2r, eta=eta_max).
 *   - ExtendPoint: step min(eta, |p_rand - p_nearest|) toward p_rand.
 *   - TraversabilityCheck: points on the segment at spacing res/2, both ends
 *     included, must all have clearance >= r_robot.
 *   - InSamplingBoundary: the map's bounding rectangle.
 *   - VoxelDownsample: voxels of side rho anchored at the map origin; the
 *     representative of a voxel is the first tree node that fell into it.
 *   - Termination: stop once a round of N_sampling attempts adds at most
 *     eps_gain new voxels (Remark 4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double x, y; } pt2;

static uint64_t rng_next(uint64_t *s) {
    /* splitmix64 (Steele, Lea, Flood 2014) */
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double rng_unit(uint64_t *s) { return (double)(rng_next(s) >> 11) * (1.0 / 9007199254740992.0); }

typedef struct {
    const float *clr;   /* per-cell clearance in metres (precomputed lookup table) */
    int W, H;
    double res;
} mapv;

/* MinDistToObstacle: table lookup at the cell containing (x, y); outside the map = 0 */
static double clearance(const mapv *m, double x, double y) {
    int cx = (int)floor(x / m->res), cy = (int)floor(y / m->res);
    if (cx < 0 || cy < 0 || cx >= m->W || cy >= m->H) return 0.0;
    return (double)m->clr[(size_t)cy * m->W + cx];
}

/* ---- spatial hash of tree nodes for exact NearestNode ---- */
typedef struct {
    int bw, bh;
    double bsize;
    int *head;   /* bucket -> first node */
    int *next;   /* node -> next node in bucket */
    pt2 *pts;
    int n, cap;
} tree;

static int tree_add(tree *t, pt2 p) {
    if (t->n == t->cap) {
        int nc = t->cap ? t->cap * 2 : 4096;
        pt2 *np = (pt2 *)realloc(t->pts, sizeof(pt2) * nc);
        int *nn = (int *)realloc(t->next, sizeof(int) * nc);
        if (!np || !nn) return -1;
        t->pts = np; t->next = nn; t->cap = nc;
    }
    int bx = (int)(p.x / t->bsize), by = (int)(p.y / t->bsize);
    if (bx < 0) bx = 0; if (bx >= t->bw) bx = t->bw - 1;
    if (by < 0) by = 0; if (by >= t->bh) by = t->bh - 1;
    int b = by * t->bw + bx;
    t->pts[t->n] = p;
    t->next[t->n] = t->head[b];
    t->head[b] = t->n;
    return t->n++;
}

static void scan_bucket(const tree *t, int x, int y, pt2 q, int *best, double *best2) {
    if (x < 0 || y < 0 || x >= t->bw || y >= t->bh) return;
    for (int i = t->head[y * t->bw + x]; i >= 0; i = t->next[i]) {
        double ex = t->pts[i].x - q.x, ey = t->pts[i].y - q.y;
        double d2 = ex * ex + ey * ey;
        if (d2 < *best2 || (d2 == *best2 && i < *best)) { *best2 = d2; *best = i; }
    }
}

/* NearestNode: exact nearest tree node, searching bucket rings outward */
static int tree_nearest(const tree *t, pt2 q) {
    int bx = (int)(q.x / t->bsize), by = (int)(q.y / t->bsize);
    if (bx < 0) bx = 0; if (bx >= t->bw) bx = t->bw - 1;
    if (by < 0) by = 0; if (by >= t->bh) by = t->bh - 1;
    int best = -1;
    double best2 = INFINITY;
    int maxr = t->bw > t->bh ? t->bw : t->bh;
    for (int r = 0; r <= maxr; ++r) {
        /* every point in ring r is more than (r-1)*bsize away */
        if (best >= 0) {
            double lo = (r - 1) * t->bsize;
            if (lo > 0 && lo * lo > best2) break;
        }
        if (r == 0) { scan_bucket(t, bx, by, q, &best, &best2); continue; }
        for (int d = -r; d <= r; ++d) {
            scan_bucket(t, bx + d, by - r, q, &best, &best2);
            scan_bucket(t, bx + d, by + r, q, &best, &best2);
        }
        for (int d = -r + 1; d <= r - 1; ++d) {
            scan_bucket(t, bx - r, by + d, q, &best, &best2);
            scan_bucket(t, bx + r, by + d, q, &best, &best2);
        }
    }
    return best;
}

/*
 * Runs Algorithm 1 from p0 and writes the voxel representatives (in order of
 * first insertion) to xy_out as (x, y) pairs in metres, map origin at (0, 0).
 * Returns the number of hypotheses written (<= cap), or -1 on bad input /
 * allocation failure.  *n_nodes_out receives the final tree size and
 * *n_rounds_out the number of rounds run.
 */
int wl_rrt_sample(const float *clr, int W, int H, double res, double p0x, double p0y,
                  double rho, double eta_max, double r_robot, int eps_gain, uint64_t seed,
                  int max_rounds, double *xy_out, int cap, int *n_nodes_out, int *n_rounds_out) {
    if (!clr || W <= 0 || H <= 0 || !(res > 0) || !(rho > 0) || !(eta_max > 0) || !(r_robot > 0))
        return -1;
    mapv m = {clr, W, H, res};
    double Wm = W * res, Hm = H * res;
    tree t;
    memset(&t, 0, sizeof t);
    t.bsize = eta_max > rho ? eta_max : rho;
    t.bw = (int)ceil(Wm / t.bsize) + 1;
    t.bh = (int)ceil(Hm / t.bsize) + 1;
    t.head = (int *)malloc(sizeof(int) * (size_t)t.bw * t.bh);
    int vw = (int)ceil(Wm / rho) + 1, vh = (int)ceil(Hm / rho) + 1;
    int *voxel = (int *)malloc(sizeof(int) * (size_t)vw * vh);
    int *reps = NULL;
    int n_reps = 0, reps_cap = 0;
    if (!t.head || !voxel) { free(t.head); free(voxel); return -1; }
    for (size_t i = 0; i < (size_t)t.bw * t.bh; ++i) t.head[i] = -1;
    for (size_t i = 0; i < (size_t)vw * vh; ++i) voxel[i] = -1;

    uint64_t s = seed;
    pt2 p0 = {p0x, p0y};
    int rc = 0;
    #define ADD_NODE(P)                                                                   \
        do {                                                                              \
            int id_ = tree_add(&t, (P));                                                  \
            if (id_ < 0) { rc = -1; goto done; }                                          \
            int vx_ = (int)floor((P).x / rho), vy_ = (int)floor((P).y / rho);             \
            int *slot_ = &voxel[(size_t)vy_ * vw + vx_];                                  \
            if (*slot_ < 0) {                                                             \
                *slot_ = id_;                                                             \
                if (n_reps == reps_cap) {                                                 \
                    reps_cap = reps_cap ? reps_cap * 2 : 1024;                            \
                    int *nr_ = (int *)realloc(reps, sizeof(int) * reps_cap);              \
                    if (!nr_) { rc = -1; goto done; }                                     \
                    reps = nr_;                                                           \
                }                                                                         \
                reps[n_reps++] = id_;                                                     \
            }                                                                             \
        } while (0)

    ADD_NODE(p0);
    double n_samp_d = ceil((double)W * H * res * res / (rho * rho));
    long n_sampling = (long)n_samp_d;
    int rounds = 0;
    int last = 0;
    for (;;) {
        for (long it = 0; it < n_sampling; ++it) {
            pt2 pr = {rng_unit(&s) * Wm, rng_unit(&s) * Hm};
            int ni = tree_nearest(&t, pr);
            pt2 pn = t.pts[ni];
            double d = clearance(&m, pn.x, pn.y);
            double eta;
            if (d >= 2.0 * r_robot) eta = eta_max;
            else if (d <= r_robot) eta = r_robot;
            else eta = r_robot + (eta_max - r_robot) * (d - r_robot) / r_robot;
            double vx = pr.x - pn.x, vy = pr.y - pn.y;
            double L = sqrt(vx * vx + vy * vy);
            if (!(L > 0)) continue;
            double step = eta < L ? eta : L;
            pt2 pnew = {pn.x + vx / L * step, pn.y + vy / L * step};
            if (!(pnew.x >= 0 && pnew.y >= 0 && pnew.x < Wm && pnew.y < Hm)) continue;
            int nseg = (int)ceil(step / (0.5 * res));
            int ok = 1;
            for (int k = 0; k <= nseg && ok; ++k) {
                double a = nseg ? (double)k / nseg : 0.0;
                double qx = pn.x + (pnew.x - pn.x) * a, qy = pn.y + (pnew.y - pn.y) * a;
                if (clearance(&m, qx, qy) < r_robot) ok = 0;
            }
            if (!ok) continue;
            ADD_NODE(pnew);
        }
        ++rounds;
        int gain = n_reps - last;
        last = n_reps;
        if (gain <= eps_gain || rounds >= max_rounds) break;
    }
    {
        int n_out = n_reps < cap ? n_reps : cap;
        for (int i = 0; i < n_out; ++i) {
            xy_out[2 * i] = t.pts[reps[i]].x;
            xy_out[2 * i + 1] = t.pts[reps[i]].y;
        }
        rc = n_out;
        if (n_nodes_out) *n_nodes_out = t.n;
        if (n_rounds_out) *n_rounds_out = rounds;
    }
done:
    #undef ADD_NODE
    free(t.head); free(t.next); free(t.pts); free(voxel); free(reps);
    return rc;
}

