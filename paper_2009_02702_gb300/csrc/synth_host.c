/*
 * synth_host.c -- seeded synthetic segmentation volumes (host side).
 *
 * Input generation only: no Mixture Graph arithmetic lives here.  The same
 * integer Voronoi rule is implemented by synth_dev.cu for the GPU, so a volume
 * generated on either side is identical bit for bit.
 *
 * Voronoi rule (all integers, exact): voxel (x, y, z) has the doubled centre
 * (2x+1, 2y+1, 2z+1); seed i sits at the doubled point s_i.  With the axis
 * metric m = (mx, my, mz) the squared distance is
 *     d_i = mx*(2x+1-sx)^2 + my*(2y+1-sy)^2 + mz*(2z+1-sz)^2
 * and the voxel takes the seed minimising d_i / W_i (W_i >= 1 an integer
 * weight), ties going to the lowest index: seed i replaces the current best j
 * when d_i * W_j < d_j * W_i.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* The ex x ey x ez block of the volume starting at voxel (x0, y0, z0),
 * x-fastest, every voxel tested against every seed (the rule as stated). */
void mgs_voronoi_block_brute(int64_t x0, int64_t y0, int64_t z0, int64_t ex, int64_t ey, int64_t ez,
                             const int64_t *seeds2, const int64_t *weight, int64_t K, const int64_t *metric,
                             int out_bytes, void *out)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < ez; z++) {
        for (int64_t y = 0; y < ey; y++) {
            for (int64_t x = 0; x < ex; x++) {
                int64_t px = 2 * (x0 + x) + 1, py = 2 * (y0 + y) + 1, pz = 2 * (z0 + z) + 1;
                int64_t best = 0, bd = -1, bw = 1;
                for (int64_t i = 0; i < K; i++) {
                    int64_t dx = px - seeds2[3 * i], dy = py - seeds2[3 * i + 1], dz = pz - seeds2[3 * i + 2];
                    int64_t d = metric[0] * dx * dx + metric[1] * dy * dy + metric[2] * dz * dz;
                    int64_t w = weight[i];
                    if (bd < 0 || d * bw < bd * w) { best = i; bd = d; bw = w; }
                }
                int64_t v = (z * ey + y) * ex + x;
                if (out_bytes == 2) ((uint16_t *)out)[v] = (uint16_t)best;
                else ((uint32_t *)out)[v] = (uint32_t)best;
            }
        }
    }
}

/* Squared metric distance from seed coordinate s to the nearest (mode 0) or
 * farthest (mode 1) of the doubled centres lo..hi along one axis. */
static int64_t axis_bound(int64_t s, int64_t lo, int64_t hi, int mode)
{
    int64_t a = s - lo < 0 ? lo - s : s - lo, b = s - hi < 0 ? hi - s : s - hi;
    if (mode == 1) return a > b ? a * a : b * b;
    if (s >= lo && s <= hi) return 0;
    return a < b ? a * a : b * b;
}

#define MGS_TILE 16

/* The same block, tile by tile: for a tile of voxels, seed i's ratio d_i/W_i
 * at any voxel lies in [lo_i/W_i, hi_i/W_i] (nearest / farthest centre of the
 * tile).  With j the seed of the smallest hi_j/W_j, every voxel's best ratio is
 * at most hi_j/W_j, so a seed with lo_i/W_i > hi_j/W_j is strictly worse than
 * the best everywhere in the tile: it can neither win nor tie.  The remaining
 * seeds, in index order, go through the rule as stated, which therefore picks
 * the same seed as the brute force for every voxel. */
void mgs_voronoi_block(int64_t x0, int64_t y0, int64_t z0, int64_t ex, int64_t ey, int64_t ez,
                       const int64_t *seeds2, const int64_t *weight, int64_t K, const int64_t *metric,
                       int out_bytes, void *out)
{
    int64_t tx = (ex + MGS_TILE - 1) / MGS_TILE, ty = (ey + MGS_TILE - 1) / MGS_TILE;
    int64_t tz = (ez + MGS_TILE - 1) / MGS_TILE;
    int64_t ntiles = tx * ty * tz;
    #pragma omp parallel
    {
        int64_t *cand = (int64_t *)malloc((size_t)(K > 0 ? K : 1) * sizeof(int64_t));
        int64_t *lob = (int64_t *)malloc((size_t)(K > 0 ? K : 1) * sizeof(int64_t));
        #pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < ntiles; t++) {
            int64_t bx = (t % tx) * MGS_TILE, by = ((t / tx) % ty) * MGS_TILE, bz = (t / (tx * ty)) * MGS_TILE;
            int64_t wx = ex - bx < MGS_TILE ? ex - bx : MGS_TILE;
            int64_t wy = ey - by < MGS_TILE ? ey - by : MGS_TILE;
            int64_t wz = ez - bz < MGS_TILE ? ez - bz : MGS_TILE;
            int64_t lo[3] = {2 * (x0 + bx) + 1, 2 * (y0 + by) + 1, 2 * (z0 + bz) + 1};
            int64_t hi[3] = {lo[0] + 2 * (wx - 1), lo[1] + 2 * (wy - 1), lo[2] + 2 * (wz - 1)};
            int64_t j = -1, hj = 0, wj = 1;
            for (int64_t i = 0; i < K; i++) {
                int64_t h = 0, l = 0;
                for (int k = 0; k < 3; k++) {
                    h += metric[k] * axis_bound(seeds2[3 * i + k], lo[k], hi[k], 1);
                    l += metric[k] * axis_bound(seeds2[3 * i + k], lo[k], hi[k], 0);
                }
                lob[i] = l;
                if (j < 0 || h * wj < hj * weight[i]) { j = i; hj = h; wj = weight[i]; }
            }
            int64_t nc = 0;
            for (int64_t i = 0; i < K; i++)
                if (!(lob[i] * wj > hj * weight[i])) cand[nc++] = i;
            for (int64_t z = bz; z < bz + wz; z++)
            for (int64_t y = by; y < by + wy; y++)
            for (int64_t x = bx; x < bx + wx; x++) {
                int64_t px = 2 * (x0 + x) + 1, py = 2 * (y0 + y) + 1, pz = 2 * (z0 + z) + 1;
                int64_t best = 0, bd = -1, bw = 1;
                for (int64_t c = 0; c < nc; c++) {
                    int64_t i = cand[c];
                    int64_t dx = px - seeds2[3 * i], dy = py - seeds2[3 * i + 1], dz = pz - seeds2[3 * i + 2];
                    int64_t d = metric[0] * dx * dx + metric[1] * dy * dy + metric[2] * dz * dz;
                    int64_t w = weight[i];
                    if (bd < 0 || d * bw < bd * w) { best = i; bd = d; bw = w; }
                }
                int64_t v = (z * ey + y) * ex + x;
                if (out_bytes == 2) ((uint16_t *)out)[v] = (uint16_t)best;
                else ((uint32_t *)out)[v] = (uint32_t)best;
            }
        }
        free(cand);
        free(lob);
    }
}

void mgs_voronoi(int64_t nx, int64_t ny, int64_t nz, const int64_t *seeds2, const int64_t *weight,
                 int64_t K, const int64_t *metric, int out_bytes, void *out)
{
    mgs_voronoi_block(0, 0, 0, nx, ny, nz, seeds2, weight, K, metric, out_bytes, out);
}

/*
 * Non-overlapping random cylinders (fibre-composite-like volume).
 * Cylinder k = 1..K is tried up to T times with pose draws rnd[k-1][t][0..7]:
 *   radius  = r0 + (r1-r0)*u0,  length = l0 + (l1-l0)*u1,
 *   axis    = (g2, g3, g4) normalised (Gaussian draws),
 *   centre  = (u5*nx, u6*ny, u7*nz).
 * A voxel centre v+1/2 is inside when its axial offset |t| <= length/2 and its
 * squared distance from the axis <= radius^2.  A pose is accepted when every
 * inside voxel is background (0); then all are painted k.  When every try
 * fails, the last pose paints only its background voxels.  A cylinder left
 * with no voxel takes the first background voxel at or after a drawn start
 * position (rnd[..][T-1][5..7]).  Returns the number of background voxels.
 */
typedef struct { double c[3], d[3], r2, h; } cyl_pose;

static void make_pose(const double *u, double r0, double r1, double l0, double l1,
                      int64_t nx, int64_t ny, int64_t nz, cyl_pose *p)
{
    double r = r0 + (r1 - r0) * u[0];
    double len = l0 + (l1 - l0) * u[1];
    double g[3] = {u[2], u[3], u[4]};
    double n = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(n > 1e-12)) { g[0] = 0; g[1] = 0; g[2] = 1; n = 1; }
    for (int k = 0; k < 3; k++) p->d[k] = g[k] / n;
    p->c[0] = u[5] * (double)nx; p->c[1] = u[6] * (double)ny; p->c[2] = u[7] * (double)nz;
    p->r2 = r * r;
    p->h = 0.5 * len;
}

/* mode 0: count non-background inside voxels; mode 1: paint all inside voxels;
 * mode 2: paint inside background voxels; mode 3: count all inside voxels.
 * Returns the count (modes 0, 3) or the number painted. */
static int64_t raster(const cyl_pose *p, int64_t nx, int64_t ny, int64_t nz, uint16_t *vol,
                      uint16_t id, int mode)
{
    double rad = sqrt(p->r2);
    double lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        double e = p->h * fabs(p->d[k]) + rad + 1.0;
        lo[k] = p->c[k] - e; hi[k] = p->c[k] + e;
    }
    int64_t z0 = (int64_t)floor(lo[2]), z1 = (int64_t)ceil(hi[2]);
    int64_t y0 = (int64_t)floor(lo[1]), y1 = (int64_t)ceil(hi[1]);
    if (z0 < 0) z0 = 0; if (z1 > nz - 1) z1 = nz - 1;
    if (y0 < 0) y0 = 0; if (y1 > ny - 1) y1 = ny - 1;
    int64_t n = 0;
    const double *d = p->d;
    for (int64_t z = z0; z <= z1; z++) {
        for (int64_t y = y0; y <= y1; y++) {
            /* point P(x) = P0 + x*ex relative to the centre */
            double P0[3] = {0.5 - p->c[0], (double)y + 0.5 - p->c[1], (double)z + 0.5 - p->c[2]};
            double t0 = P0[0] * d[0] + P0[1] * d[1] + P0[2] * d[2];
            double td = d[0];
            /* axial: |t0 + td*x| <= h */
            double xa, xb;
            if (fabs(td) < 1e-12) {
                if (fabs(t0) > p->h) continue;
                xa = -1e300; xb = 1e300;
            } else {
                double u1 = (-p->h - t0) / td, u2 = (p->h - t0) / td;
                xa = u1 < u2 ? u1 : u2; xb = u1 < u2 ? u2 : u1;
            }
            /* radial: |P|^2 - t^2 <= r2, a quadratic A x^2 + B x + C <= 0 */
            double A = 1.0 - td * td;
            double B = 2.0 * (P0[0] - t0 * td);
            double Cq = P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2] - t0 * t0 - p->r2;
            double ra, rb;
            if (A < 1e-12) {
                if (Cq > 0) continue;
                ra = -1e300; rb = 1e300;
            } else {
                double disc = B * B - 4 * A * Cq;
                if (disc < 0) continue;
                double sq = sqrt(disc);
                ra = (-B - sq) / (2 * A); rb = (-B + sq) / (2 * A);
            }
            double a = xa > ra ? xa : ra, b = xb < rb ? xb : rb;
            if (a > b) continue;
            int64_t xs = (int64_t)ceil(a - 1e-9), xe = (int64_t)floor(b + 1e-9);
            if (xs < 0) xs = 0;
            if (xe > nx - 1) xe = nx - 1;
            for (int64_t x = xs; x <= xe; x++) {
                /* exact membership test on the voxel centre */
                double P[3] = {P0[0] + (double)x, P0[1], P0[2]};
                double t = P[0] * d[0] + P[1] * d[1] + P[2] * d[2];
                if (fabs(t) > p->h) continue;
                double rr = P[0] * P[0] + P[1] * P[1] + P[2] * P[2] - t * t;
                if (rr > p->r2) continue;
                uint16_t *vp = vol + (z * ny + y) * nx + x;
                if (mode == 0) { if (*vp) n++; }
                else if (mode == 3) n++;
                else if (mode == 1) { *vp = id; n++; }
                else if (*vp == 0) { *vp = id; n++; }
            }
        }
    }
    return n;
}

int64_t mgs_cylinders(int64_t nx, int64_t ny, int64_t nz, int64_t K, int64_t T, const double *rnd,
                      double r0, double r1, double l0, double l1, uint16_t *vol)
{
    int64_t V = nx * ny * nz;
    memset(vol, 0, (size_t)V * sizeof(uint16_t));
    /* The tries of one cylinder only read the volume, so a group of them is
     * tested in parallel; the first accepted try in order wins, exactly as a
     * serial scan of the tries would choose. */
    enum { G = 16 };
    for (int64_t k = 1; k <= K; k++) {
        const double *base = rnd + (k - 1) * T * 8;
        cyl_pose p;
        int64_t painted = 0;
        int done = 0;
        for (int64_t t0 = 0; t0 < T && !done; t0 += G) {
            int64_t n = T - t0 < G ? T - t0 : G;
            int64_t blocked[G], inside[G];
            #pragma omp parallel for schedule(dynamic, 1)
            for (int64_t j = 0; j < n; j++) {
                cyl_pose q;
                make_pose(base + (t0 + j) * 8, r0, r1, l0, l1, nx, ny, nz, &q);
                blocked[j] = raster(&q, nx, ny, nz, vol, 0, 0);
                inside[j] = blocked[j] == 0 ? raster(&q, nx, ny, nz, vol, 0, 3) : 0;
            }
            for (int64_t j = 0; j < n && !done; j++) {
                make_pose(base + (t0 + j) * 8, r0, r1, l0, l1, nx, ny, nz, &p);
                if (blocked[j] == 0 && inside[j] > 0) {
                    painted = raster(&p, nx, ny, nz, vol, (uint16_t)k, 1);
                    done = 1;
                }
            }
        }
        if (!done) painted = raster(&p, nx, ny, nz, vol, (uint16_t)k, 2);
        if (painted == 0) {
            const double *u = base + (T - 1) * 8;
            int64_t start = (int64_t)(u[5] * (double)V);
            if (start >= V) start = V - 1;
            for (int64_t i = 0; i < V; i++) {
                int64_t j = (start + i) % V;
                if (vol[j] == 0) { vol[j] = (uint16_t)k; break; }
            }
        }
    }
    int64_t bg = 0;
    for (int64_t i = 0; i < V; i++) bg += vol[i] == 0;
    return bg;
}
