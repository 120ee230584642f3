/*
 * Noise-free depth of a synthetic scene (planes, axis-aligned boxes and facades with
 * window recesses) seen by a pinhole camera: the z-buffer of exact ray casts through
 * pixel centres.  This is input generation only; it holds none of the method's
 * arithmetic.  synth/scenes.py states the same casts in numpy; this file evaluates them
 * in the same operation order (compiled without floating-point contraction), so both
 * give the same float64 depths, and it is what Scene.render_clean calls when built.
 *
 * Camera rays: d_cam = (((x + 0.5) - cx) / fx, ((y + 0.5) - cy) / fy, 1); world ray
 * D = R d_cam (each row summed left to right), origin o = t; a hit at ray parameter lam
 * lies at camera depth lam (d_cam has z = 1).
 */
#include <math.h>
#include <stdint.h>

/* rect: axis, value, lo[2], hi[2] (the two other axes in ascending order) */
typedef struct { double axis, value, lo0, lo1, hi0, hi1; } rect_t;
/* box: lo[3], hi[3] */
typedef struct { double lo[3], hi[3]; } box_t;
/* facade: plane x (side), y range, z range, cell (z, y), window (z, y), recess depth,
 * window lattice nz x ny (bool, [iz][iy]) */
typedef struct { double x, side, y_top, y_bot, z0, z1, cz, cy, wz, wy, recess, nz, ny; } facade_t;

static void hit_rect(double *best, const double *o, const double *D, int n, const rect_t *r) {
    const int a = (int)r->axis;
    const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
    for (int i = 0; i < n; ++i) {
        const double lam = (r->value - o[a]) / D[3 * i + a];
        if (!(lam > 0.0)) continue;
        const double c0 = o[b0] + lam * D[3 * i + b0];
        if (!(c0 >= r->lo0 && c0 <= r->hi0)) continue;
        const double c1 = o[b1] + lam * D[3 * i + b1];
        if (!(c1 >= r->lo1 && c1 <= r->hi1)) continue;
        if (lam < best[i]) best[i] = lam;
    }
}

static double fmin_nan(double a, double b) { return (a != a || b != b) ? NAN : (a < b ? a : b); }
static double fmax_nan(double a, double b) { return (a != a || b != b) ? NAN : (a > b ? a : b); }

/* Slab test of the pixels of rows [y0, y1) x columns [x0, x1). */
static void hit_box(double *best, const double *o, const double *D, int W, int y0, int y1, int x0, int x1,
                    const box_t *b) {
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            const int i = y * W + x;
            double t_near = -INFINITY, t_far = INFINITY;
            for (int a = 0; a < 3; ++a) {
                const double Da = D[3 * i + a];
                double lo, hi;
                if (Da == 0.0) {
                    const int inside = o[a] >= b->lo[a] && o[a] <= b->hi[a];
                    lo = inside ? -INFINITY : INFINITY;
                    hi = inside ? INFINITY : -INFINITY;
                } else {
                    const double inv = 1.0 / Da;
                    const double t1 = (b->lo[a] - o[a]) * inv, t2 = (b->hi[a] - o[a]) * inv;
                    lo = fmin_nan(t1, t2);
                    hi = fmax_nan(t1, t2);
                }
                t_near = fmax_nan(t_near, lo);
                t_far = fmin_nan(t_far, hi);
            }
            if (t_near <= t_far && t_near > 0.0 && t_near < best[i]) best[i] = t_near;
        }
}

static void hit_facade(double *best, const double *o, const double *D, int n, const facade_t *f,
                       const uint8_t *windows) {
    const int nz = (int)f->nz, ny = (int)f->ny;
    for (int i = 0; i < n; ++i) {
        const double Dx = D[3 * i], Dy = D[3 * i + 1], Dz = D[3 * i + 2];
        if (!((f->x - o[0]) * Dx > 0.0)) continue;
        const double lam = (f->x - o[0]) / Dx;
        const double y = o[1] + lam * Dy, z = o[2] + lam * Dz;
        const int ok = y >= f->y_top && y <= f->y_bot && z >= f->z0 && z <= f->z1;
        double depth = ok ? lam : INFINITY;
        const double iz = floor((z - f->z0) / f->cz), iy = floor((y - f->y_top) / f->cy);
        const int inside_grid = ok && iz >= 0.0 && iz < (double)nz && iy >= 0.0 && iy < (double)ny;
        if (inside_grid && windows[(int64_t)iz * ny + (int64_t)iy]) {
            const double izc = iz, iyc = iy;
            const double wz0 = (f->z0 + izc * f->cz) + 0.5 * (f->cz - f->wz);
            const double wy0 = (f->y_top + iyc * f->cy) + 0.5 * (f->cy - f->wy);
            const double wz1 = wz0 + f->wz, wy1 = wy0 + f->wy;
            if (z > wz0 && z < wz1 && y > wy0 && y < wy1) {
                const double xb = f->x + f->side * f->recess;
                const double lam_b = (xb - o[0]) / Dx;
                double lam_exit = INFINITY;
                const double ob[2] = {o[1], o[2]}, Db[2] = {Dy, Dz}, lo[2] = {wy0, wz0}, hi[2] = {wy1, wz1};
                for (int k = 0; k < 2; ++k) {
                    const double t_hi = Db[k] > 0.0 ? (hi[k] - ob[k]) / Db[k] : INFINITY;
                    const double t_lo = Db[k] < 0.0 ? (lo[k] - ob[k]) / Db[k] : INFINITY;
                    lam_exit = fmin_nan(lam_exit, fmin_nan(t_hi, t_lo));
                }
                depth = fmin_nan(lam_b, lam_exit);
            }
        }
        if (depth < best[i]) best[i] = depth;
    }
}

/* Noise-free depth [H][W] (0 where nothing is hit within d_max).  T: camera -> world
 * 4x4 row-major.  box_win: per box the pixel window (y0, y1, x0, x1) that holds its
 * projection, or y0 = -1 for the whole image, or y0 == y1 for none.  ray_buf: scratch
 * of 3 W H doubles. */
void raycast_depth(int W, int H, double fx, double fy, double cx, double cy, const double *T, int n_rect,
                   const rect_t *rects, int n_box, const box_t *boxes, const int32_t *box_win, int n_fac,
                   const facade_t *facades, const uint8_t *windows, double d_max, double *ray_buf, double *out) {
    const double o[3] = {T[3], T[7], T[11]};
    double *D = ray_buf;
    const int n = W * H;
    for (int y = 0; y < H; ++y) {
        const double dy = (((double)y + 0.5) - cy) / fy;
        for (int x = 0; x < W; ++x) {
            const double dx = (((double)x + 0.5) - cx) / fx;
            double *d = D + 3 * (y * W + x);
            for (int r = 0; r < 3; ++r) d[r] = (T[4 * r] * dx + T[4 * r + 1] * dy) + T[4 * r + 2] * 1.0;
        }
    }
    for (int i = 0; i < n; ++i) out[i] = INFINITY;
    for (int k = 0; k < n_rect; ++k) hit_rect(out, o, D, n, rects + k);
    for (int k = 0; k < n_box; ++k) {
        const int32_t *w = box_win + 4 * k;
        if (w[0] < 0) hit_box(out, o, D, W, 0, H, 0, W, boxes + k);
        else if (w[0] < w[1]) hit_box(out, o, D, W, w[0], w[1], w[2], w[3], boxes + k);
    }
    const uint8_t *win = windows;
    for (int k = 0; k < n_fac; ++k) {
        hit_facade(out, o, D, n, facades + k, win);
        win += (int64_t)facades[k].nz * (int64_t)facades[k].ny;
    }
    for (int i = 0; i < n; ++i)
        if (!(out[i] <= d_max)) out[i] = 0.0;
}
