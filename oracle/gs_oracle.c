/*
 * FP64 CPU oracle for the 3D Gaussian splatting forward hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this code.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * It is written as the plain definition of each step, in double precision,
 * with no blocking, fusion or reordering:
 *
 *   preprocess        Section II-B (1): cull the Gaussians outside the view,
 *                     project each 3D Gaussian to a 2D splat with colour and
 *                     depth.  The projection is the EWA splatting of the
 *                     original 3DGS renderer that the paper builds on (cited
 *                     in Sections II-A and II-B): Sigma = R S S^T R^T,
 *                     Sigma' = J W Sigma W^T J^T + 0.3 I, conic = Sigma'^-1,
 *                     radius = ceil(3 sqrt(lambda_max)), colour from degree-3
 *                     real spherical harmonics.
 *   duplicate + sort  Section II-B (1): each splat is replicated for every
 *                     16x16 tile its rectangle touches and the replicas are
 *                     sorted by depth within each tile; the key is
 *                     (tile id << 32 | FP32 depth bits), ties keep the
 *                     emission order (Gaussian id, then row-major tile).
 *   ranges            Section II-B (2) and Algorithm 1: per tile the [start,
 *                     end) range of its replicas in the sorted list.
 *   render            Eq. 1 with the kernel's alpha of Algorithm 1 and the
 *                     per-pixel rules of the Appendix B kernels:
 *                     power = -(a dx^2 + c dy^2)/2 - b dx dy, skip power > 0,
 *                     alpha = min(0.99, o exp(power)), skip alpha < 1/255,
 *                     stop (without blending) once T (1 - alpha) < 1e-4,
 *                     out = C + T bg, final_T = T, n_contrib = 1-based list
 *                     position of the last blended Gaussian.
 *
 * The one FP32 quantity is the depth that enters the sort key and the near
 * plane test: the paper's kernels compute in float32 (Section IV-B), the key
 * is an integer code taken from that float, and both sides must take the same
 * decision, so the oracle evaluates it as the correctly rounded expression
 * fmaf(V22, mz, fmaf(V21, my, fmaf(V20, mx, V23))).
 *
 * Integer decisions made from floating point (radius, tile rectangle) are
 * taken in FP64; the oracle also reports each decision's distance to its
 * boundary so that a comparison can tell a genuine mismatch from an FP32
 * rounding flip.  The same holds per pixel for the alpha and transmittance
 * thresholds of the blend.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TILE 16
#define NEAR_Z 0.2f
#define DILATION 0.3
#define FRUSTUM_SLACK 1.3
#define LAMBDA_FLOOR 0.1
#define ALPHA_MAX 0.99
#define ALPHA_MIN (1.0 / 255.0)
#define T_MIN 1e-4

typedef struct {
    double V[4][4];          /* world -> camera, row-major */
    float V32[4][4];         /* the same matrix as given, in float */
    double fx, fy, cx, cy, tan_fovx, tan_fovy;
    int width, height, tiles_x, tiles_y;
} camera_t;

/* cam: viewmat[16] (row-major), fx, fy, cx, cy, width, height, tan_fovx, tan_fovy */
static void read_camera(const float *cam, camera_t *c) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            c->V32[i][j] = cam[4 * i + j];
            c->V[i][j] = (double)cam[4 * i + j];
        }
    c->fx = cam[16];
    c->fy = cam[17];
    c->cx = cam[18];
    c->cy = cam[19];
    c->width = (int)cam[20];
    c->height = (int)cam[21];
    c->tan_fovx = cam[22];
    c->tan_fovy = cam[23];
    c->tiles_x = (c->width + TILE - 1) / TILE;
    c->tiles_y = (c->height + TILE - 1) / TILE;
}

/* ---------------------------------------------------------------------------
 * Real spherical harmonics, orthonormal on the unit sphere, with the
 * Condon-Shortley phase, ordered k = l^2 + l + m (m = -l..l).  Built from the
 * textbook definition: associated Legendre functions by their three-term
 * recurrence and the normalisation sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!).
 * ------------------------------------------------------------------------- */
static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

/* P_l^m(x) for m >= 0, including the (-1)^m Condon-Shortley factor. */
static double assoc_legendre(int l, int m, double x) {
    double somx2 = sqrt(fmax(0.0, (1.0 - x) * (1.0 + x)));
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * somx2;
    if (l == m) return pmm;
    double pmmp1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pmmp1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * x * pmmp1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pmmp1;
        pmmp1 = pll;
    }
    return pll;
}

double oracle_sh_basis(int l, int m, double x, double y, double z) {
    int am = m < 0 ? -m : m;
    double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
    double P = assoc_legendre(l, am, z);
    double phi = atan2(y, x);
    if (m == 0) return K * P;
    if (m > 0) return sqrt(2.0) * K * cos(m * phi) * P;
    return sqrt(2.0) * K * sin(am * phi) * P;
}

/* ---------------------------------------------------------------------------
 * Preprocess (Section II-B (1)).
 * ------------------------------------------------------------------------- */
static double dist_to_int(double v) { return fabs(v - nearbyint(v)); }

/* Distance (in the units of v) from v to the nearest multiple of `step` that
 * changes clamp(floor(v / step), 0, hi); a huge value if none is near. */
static double rect_edge_dist(double v, double step, int hi) {
    double k = nearbyint(v / step);
    if (k < 1.0 || k > (double)hi) return 1e30;
    return fabs(v - k * step);
}

static int clampi(long long v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : (int)v); }

/*
 * Inputs are the float32 scene arrays (SoA) and the camera record.
 * Outputs (all [n]-major, caller-allocated):
 *   xy[2n]          pixel-space mean
 *   cov2d[3n]       Sigma' entries (s00, s01, s11), dilation included
 *   conic[3n]       Sigma'^-1 entries (a, b, c)
 *   opacity[n]      sigmoid(logit)
 *   rgb[3n]         SH colour + 0.5, clamped at 0
 *   depth[n]        view-space z in FP64
 *   depth32[n]      view-space z as the FP32 sort-key value
 *   radius[n]       ceil(3 sqrt(lambda_max)); 0 for culled Gaussians
 *   rect[4n]        tile rectangle x0, y0, x1, y1 (exclusive max)
 *   tiles[n]        (x1 - x0)(y1 - y0); 0 for culled Gaussians
 *   rad_dist[n]     |3 sqrt(lambda_max) - nearest integer|
 *   edge_dist[n]    min over the four rectangle edges of the distance (in
 *                   pixels) to the nearest edge-changing tile boundary
 * Returns the number of visible Gaussians.
 */
int64_t oracle_preprocess(int64_t n, const float *means, const float *log_scales, const float *quats,
                          const float *opacity_logits, const float *sh, int sh_degree, const float *cam_rec,
                          double *xy, double *cov2d, double *conic, double *opacity, double *rgb,
                          double *depth, float *depth32, int32_t *radius, int32_t *rect, int32_t *tiles,
                          double *rad_dist, double *edge_dist) {
    camera_t cam;
    read_camera(cam_rec, &cam);
    /* camera centre in world space: -R^T t */
    double campos[3];
    for (int i = 0; i < 3; ++i) {
        campos[i] = 0.0;
        for (int j = 0; j < 3; ++j) campos[i] -= cam.V[j][i] * cam.V[j][3];
    }
    int64_t visible = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 4096) reduction(+ : visible)
#endif
    for (int64_t g = 0; g < n; ++g) {
        const float *mf = means + 3 * g;
        double m[3] = {mf[0], mf[1], mf[2]};
        /* defaults for a culled Gaussian */
        xy[2 * g] = xy[2 * g + 1] = 0.0;
        for (int k = 0; k < 3; ++k) cov2d[3 * g + k] = conic[3 * g + k] = rgb[3 * g + k] = 0.0;
        opacity[g] = 0.0;
        radius[g] = 0;
        tiles[g] = 0;
        for (int k = 0; k < 4; ++k) rect[4 * g + k] = 0;
        rad_dist[g] = edge_dist[g] = 1e30;

        /* view-space position */
        double t[3];
        for (int i = 0; i < 3; ++i) t[i] = cam.V[i][0] * m[0] + cam.V[i][1] * m[1] + cam.V[i][2] * m[2] + cam.V[i][3];
        depth[g] = t[2];
        float z32 = fmaf(cam.V32[2][2], mf[2], fmaf(cam.V32[2][1], mf[1], fmaf(cam.V32[2][0], mf[0], cam.V32[2][3])));
        depth32[g] = z32;
        if (z32 <= NEAR_Z) continue; /* near-plane cull */

        /* 3D covariance Sigma = R S S^T R^T from the normalised quaternion */
        const float *qf = quats + 4 * g;
        double qn = sqrt((double)qf[0] * qf[0] + (double)qf[1] * qf[1] + (double)qf[2] * qf[2] + (double)qf[3] * qf[3]);
        double w = qf[0] / qn, x = qf[1] / qn, y = qf[2] / qn, z = qf[3] / qn;
        double R[3][3] = {
            {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},
            {2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)},
            {2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)},
        };
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = exp((double)log_scales[3 * g + k]);
        double Sigma[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += R[i][k] * s[k] * s[k] * R[j][k];
                Sigma[i][j] = acc;
            }

        /* EWA: Jacobian of the perspective map at the (frustum-clamped) mean */
        double tz = t[2];
        double limx = FRUSTUM_SLACK * cam.tan_fovx, limy = FRUSTUM_SLACK * cam.tan_fovy;
        double txc = fmin(limx, fmax(-limx, t[0] / tz)) * tz;
        double tyc = fmin(limy, fmax(-limy, t[1] / tz)) * tz;
        double J[2][3] = {{cam.fx / tz, 0.0, -cam.fx * txc / (tz * tz)},
                          {0.0, cam.fy / tz, -cam.fy * tyc / (tz * tz)}};
        double T[2][3]; /* J W, W = rotation part of the view matrix */
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += J[i][k] * cam.V[k][j];
                T[i][j] = acc;
            }
        double C2[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += T[i][k] * Sigma[k][l] * T[j][l];
                C2[i][j] = acc;
            }
        double s00 = C2[0][0] + DILATION, s01 = C2[0][1], s11 = C2[1][1] + DILATION;
        double det = s00 * s11 - s01 * s01;
        if (det == 0.0) continue;
        double mid = 0.5 * (s00 + s11);
        double lam1 = mid + sqrt(fmax(LAMBDA_FLOOR, mid * mid - det));
        double lam2 = mid - sqrt(fmax(LAMBDA_FLOOR, mid * mid - det));
        double rr = 3.0 * sqrt(fmax(lam1, lam2));
        int r = (int)ceil(rr);

        double px = cam.fx * t[0] / tz + cam.cx;
        double py = cam.fy * t[1] / tz + cam.cy;
        int x0 = clampi((long long)floor((px - r) / TILE), 0, cam.tiles_x);
        int y0 = clampi((long long)floor((py - r) / TILE), 0, cam.tiles_y);
        int x1 = clampi((long long)floor((px + r + TILE - 1) / TILE), 0, cam.tiles_x);
        int y1 = clampi((long long)floor((py + r + TILE - 1) / TILE), 0, cam.tiles_y);
        /* decision distances, reported even if the rectangle is empty */
        rad_dist[g] = dist_to_int(rr);
        double e = rect_edge_dist(px - r, TILE, cam.tiles_x);
        e = fmin(e, rect_edge_dist(py - r, TILE, cam.tiles_y));
        e = fmin(e, rect_edge_dist(px + r + TILE - 1, TILE, cam.tiles_x));
        e = fmin(e, rect_edge_dist(py + r + TILE - 1, TILE, cam.tiles_y));
        edge_dist[g] = e;
        if ((x1 - x0) * (y1 - y0) == 0) continue;

        /* colour: degree-<=3 SH along the viewing direction, + 0.5, clamped at 0 */
        double d[3] = {m[0] - campos[0], m[1] - campos[1], m[2] - campos[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) d[k] /= dn;
        double Y[16];
        for (int l = 0; l <= sh_degree; ++l)
            for (int mm = -l; mm <= l; ++mm) Y[l * l + l + mm] = oracle_sh_basis(l, mm, d[0], d[1], d[2]);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int k = 0; k < (sh_degree + 1) * (sh_degree + 1); ++k) acc += (double)sh[(g * 16 + k) * 3 + ch] * Y[k];
            rgb[3 * g + ch] = fmax(acc + 0.5, 0.0);
        }

        xy[2 * g] = px;
        xy[2 * g + 1] = py;
        cov2d[3 * g] = s00;
        cov2d[3 * g + 1] = s01;
        cov2d[3 * g + 2] = s11;
        conic[3 * g] = s11 / det;
        conic[3 * g + 1] = -s01 / det;
        conic[3 * g + 2] = s00 / det;
        opacity[g] = 1.0 / (1.0 + exp(-(double)opacity_logits[g]));
        radius[g] = r;
        rect[4 * g] = x0;
        rect[4 * g + 1] = y0;
        rect[4 * g + 2] = x1;
        rect[4 * g + 3] = y1;
        tiles[g] = (x1 - x0) * (y1 - y0);
        ++visible;
    }
    return visible;
}

/* ---------------------------------------------------------------------------
 * Duplicate, sort, ranges (Section II-B; Algorithm 1 "load work range").
 * ------------------------------------------------------------------------- */
typedef struct {
    uint64_t key;
    uint32_t val;
} kv_t;

static int kv_cmp(const void *pa, const void *pb) {
    const kv_t *a = (const kv_t *)pa, *b = (const kv_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    /* equal key: same tile and depth; emission order is ascending id */
    return a->val < b->val ? -1 : (a->val > b->val ? 1 : 0);
}

int64_t oracle_num_instances(int64_t n, const int32_t *tiles) {
    int64_t m = 0;
    for (int64_t g = 0; g < n; ++g) m += tiles[g];
    return m;
}

/* keys[m], vals[m], ranges[2 * num_tiles] are caller-allocated; m must equal
 * oracle_num_instances.  depth32 supplies the key's low 32 bits. */
void oracle_duplicate_sort(int64_t n, const int32_t *rect, const int32_t *tiles, const float *depth32,
                           int tiles_x, int num_tiles, int64_t m, uint64_t *keys, uint32_t *vals,
                           uint32_t *ranges) {
    kv_t *list = (kv_t *)malloc(sizeof(kv_t) * (size_t)(m > 0 ? m : 1));
    int64_t k = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (tiles[g] == 0) continue;
        uint32_t dbits;
        memcpy(&dbits, &depth32[g], 4);
        const int32_t *rc = rect + 4 * g;
        for (int y = rc[1]; y < rc[3]; ++y)
            for (int x = rc[0]; x < rc[2]; ++x) {
                uint64_t tile = (uint64_t)y * (uint64_t)tiles_x + (uint64_t)x;
                list[k].key = (tile << 32) | (uint64_t)dbits;
                list[k].val = (uint32_t)g;
                ++k;
            }
    }
    qsort(list, (size_t)k, sizeof(kv_t), kv_cmp);
    for (int64_t i = 0; i < k; ++i) {
        keys[i] = list[i].key;
        vals[i] = list[i].val;
    }
    for (int t = 0; t < 2 * num_tiles; ++t) ranges[t] = 0;
    for (int64_t i = 0; i < k; ++i) {
        uint32_t tile = (uint32_t)(list[i].key >> 32);
        if (i == 0 || (uint32_t)(list[i - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)i;
        if (i == k - 1 || (uint32_t)(list[i + 1].key >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(i + 1);
    }
    free(list);
}

/* ---------------------------------------------------------------------------
 * Per-pixel compositing (Eq. 1, Algorithm 1, Appendix B semantics).
 *
 * ids[0..len) is the pixel's front-to-back list.  Besides the colour, final
 * T and contributor index, it reports:
 *   invdepth      the inverse depth blended like a colour channel, without
 *                 background: sum over blended Gaussians of alpha T / z (the
 *                 optional output of the paper's render kernels, Appendix B)
 *   n_eval        Gaussians evaluated before the pixel stopped (the
 *                 "Gaussian-pixel evaluations" work count)
 *   near_count    threshold decisions (alpha < 1/255 skip, T (1 - alpha) <
 *                 1e-4 stop) whose log-space distance to the threshold is
 *                 under tau_alpha / tau_T, widened by how far a relative
 *                 rounding pos_eps of the splat's pixel coordinates can move
 *                 that distance (FP32 stores them with ulp ~ |x| 2^-24):
 *                 |d log(alpha) / d x| pos_eps (|x| + 1) + the same for y,
 *                 times alpha / (1 - alpha) for the stop decision, whose
 *                 quantity is log(1 - alpha)
 *   flip_impact   over those near decisions, the largest change of any colour
 *                 channel when that one decision is taken the other way and
 *                 the rest of the list is walked again exactly (so a flip
 *                 that moves a later stop is counted in full)
 * ------------------------------------------------------------------------- */
enum { DECIDE_ALPHA = 0, DECIDE_STOP = 1 };

typedef struct {
    double color[3];
    double invdepth;
    double T;
    int32_t n_contrib;
    int32_t n_eval;
    int32_t near_count;
    double flip_impact;
} pixel_t;

/* Growable list of near decisions: entry = 2 * list index + kind. */
typedef struct {
    int64_t *at;
    int64_t n, cap;
    int64_t local[32];
} near_list_t;

static void near_push(near_list_t *l, int64_t v) {
    if (l->n == l->cap) {
        int64_t cap = 2 * l->cap;
        int64_t *p = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        memcpy(p, l->at, sizeof(int64_t) * (size_t)l->n);
        if (l->at != l->local) free(l->at);
        l->at = p;
        l->cap = cap;
    }
    l->at[l->n++] = v;
}

/* The walk of one pixel.  flip < 0: as defined.  Otherwise the decision
 * flip = 2 i + kind (list entry i) is taken the other way: a skipped
 * Gaussian is blended with its alpha, a blended one skipped; a stop is not
 * taken, or taken there.  near (may be NULL) collects the near decisions. */
static pixel_t walk_pixel(double pxf, double pyf, const uint32_t *ids, int64_t len, const double *xy,
                          const double *conic, const double *opacity, const double *rgb, const double *depth,
                          const double *bg, double tau_alpha, double tau_T, double pos_eps, int64_t flip,
                          near_list_t *near) {
    pixel_t out;
    double T = 1.0, C[3] = {0.0, 0.0, 0.0}, D = 0.0;
    int32_t contrib = 0, last = 0;
    for (int64_t i = 0; i < len; ++i) {
        uint32_t g = ids[i];
        ++contrib;
        double dx = xy[2 * g] - pxf, dy = xy[2 * g + 1] - pyf;
        double a = conic[3 * g], b = conic[3 * g + 1], c = conic[3 * g + 2];
        double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        if (power > 0.0) continue;
        double raw = opacity[g] * exp(power);
        double alpha = fmin(ALPHA_MAX, raw);
        /* |d log(alpha) / d x_g| pos_eps (|x_g| + 1) + the same for y */
        double gx = fabs(a * dx + b * dy), gy = fabs(b * dx + c * dy);
        double pos_err = pos_eps * (gx * (fabs(xy[2 * g]) + 1.0) + gy * (fabs(xy[2 * g + 1]) + 1.0));
        if (near && raw > 0.0 && fabs(log(raw) - log(ALPHA_MIN)) < tau_alpha + pos_err)
            near_push(near, 2 * i + DECIDE_ALPHA);
        int skip = alpha < ALPHA_MIN;
        if (flip == 2 * i + DECIDE_ALPHA) skip = !skip;
        if (skip) continue;
        double Tn = T * (1.0 - alpha);
        if (near && fabs(log(Tn) - log(T_MIN)) < tau_T + pos_err * alpha / (1.0 - alpha))
            near_push(near, 2 * i + DECIDE_STOP);
        int stop = Tn < T_MIN;
        if (flip == 2 * i + DECIDE_STOP) stop = !stop;
        if (stop) break; /* stop; this Gaussian is not blended */
        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
        D += alpha * T / depth[g];
        T = Tn;
        last = contrib;
    }
    for (int ch = 0; ch < 3; ++ch) out.color[ch] = C[ch] + T * bg[ch];
    out.invdepth = D;
    out.T = T;
    out.n_contrib = last;
    out.n_eval = contrib;
    out.near_count = 0;
    out.flip_impact = 0.0;
    return out;
}

static pixel_t composite_pixel(double pxf, double pyf, const uint32_t *ids, int64_t len, const double *xy,
                               const double *conic, const double *opacity, const double *rgb, const double *depth,
                               const double *bg, double tau_alpha, double tau_T, double pos_eps) {
    near_list_t near;
    near.at = near.local;
    near.n = 0;
    near.cap = 32;
    pixel_t out = walk_pixel(pxf, pyf, ids, len, xy, conic, opacity, rgb, depth, bg, tau_alpha, tau_T, pos_eps, -1,
                             &near);
    double impact = 0.0;
    for (int64_t k = 0; k < near.n; ++k) {
        pixel_t alt = walk_pixel(pxf, pyf, ids, len, xy, conic, opacity, rgb, depth, bg, 0.0, 0.0, 0.0, near.at[k],
                                 NULL);
        for (int ch = 0; ch < 3; ++ch) impact = fmax(impact, fabs(alt.color[ch] - out.color[ch]));
    }
    out.near_count = (int32_t)near.n;
    out.flip_impact = impact;
    if (near.at != near.local) free(near.at);
    return out;
}

static void store_pixel(const pixel_t *p, int64_t pix, int64_t npix, double *out_color, double *invdepth,
                        double *final_T, int32_t *n_contrib, int32_t *n_eval, int32_t *near_count,
                        double *flip_impact) {
    for (int ch = 0; ch < 3; ++ch) out_color[ch * npix + pix] = p->color[ch];
    invdepth[pix] = p->invdepth;
    final_T[pix] = p->T;
    n_contrib[pix] = p->n_contrib;
    n_eval[pix] = p->n_eval;
    near_count[pix] = p->near_count;
    flip_impact[pix] = p->flip_impact;
}

/* Tiled render: each pixel walks its tile's range of the sorted list.
 * Rows of pixels in [row0, row1) are rendered (the rest untouched), using
 * nthreads OpenMP threads if built with OpenMP. */
void oracle_render(int width, int height, int row0, int row1, const uint32_t *ranges, const uint32_t *vals,
                   int64_t n, const double *xy, const double *conic, const double *opacity, const double *rgb,
                   const double *depth, const double *bg, double tau_alpha, double tau_T, double pos_eps,
                   int nthreads, double *out_color, double *invdepth, double *final_T, int32_t *n_contrib,
                   int32_t *n_eval, int32_t *near_count, double *flip_impact) {
    int tiles_x = (width + TILE - 1) / TILE;
    int64_t npix = (int64_t)width * height;
    (void)n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int py = row0; py < row1; ++py) {
        for (int px = 0; px < width; ++px) {
            int tile = (py / TILE) * tiles_x + px / TILE;
            uint32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
            pixel_t p = composite_pixel((double)px, (double)py, vals + s, (int64_t)e - (int64_t)s, xy, conic,
                                        opacity, rgb, depth, bg, tau_alpha, tau_T, pos_eps);
            store_pixel(&p, (int64_t)py * width + px, npix, out_color, invdepth, final_T, n_contrib, n_eval,
                        near_count, flip_impact);
        }
    }
}

/* Brute force without tile lists: for every pixel, collect every Gaussian
 * (restricted to those whose rectangle contains the pixel's tile when
 * `use_rect` is set; otherwise every Gaussian in front of the near plane with
 * a non-zero radius), order them by (FP32 depth, id) and composite.  For tiny
 * scenes only. */
static const float *g_bf_depth;
static int bf_cmp(const void *pa, const void *pb) {
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    float da = g_bf_depth[a], db = g_bf_depth[b];
    if (da != db) return da < db ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

void oracle_render_bruteforce(int width, int height, int64_t n, const int32_t *rect, const int32_t *radius,
                              const float *depth32, const double *xy, const double *conic, const double *opacity,
                              const double *rgb, const double *depth, const double *bg, int use_rect,
                              double *out_color, double *invdepth, double *final_T, int32_t *n_contrib,
                              int32_t *n_eval, int32_t *near_count, double *flip_impact) {
    int64_t npix = (int64_t)width * height;
    uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    g_bf_depth = depth32;
    for (int py = 0; py < height; ++py)
        for (int px = 0; px < width; ++px) {
            int tx = px / TILE, ty = py / TILE;
            int64_t len = 0;
            for (int64_t g = 0; g < n; ++g) {
                if (radius[g] == 0) continue;
                if (use_rect) {
                    const int32_t *rc = rect + 4 * g;
                    if (!(tx >= rc[0] && tx < rc[2] && ty >= rc[1] && ty < rc[3])) continue;
                }
                ids[len++] = (uint32_t)g;
            }
            qsort(ids, (size_t)len, sizeof(uint32_t), bf_cmp);
            pixel_t p = composite_pixel((double)px, (double)py, ids, len, xy, conic, opacity, rgb, depth, bg, 0.0,
                                        0.0, 0.0);
            store_pixel(&p, (int64_t)py * width + px, npix, out_color, invdepth, final_T, n_contrib, n_eval,
                        near_count, flip_impact);
        }
    free(ids);
}

int oracle_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
