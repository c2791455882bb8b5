/*
 * FP64 CPU oracle of the tile-binned 3D Gaussian splatting pass, its adjoint
 * and the per-Gaussian edge score.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke test and the CPU-baseline
 * leg of the benchmark load this library; the product path never does.  It
 * shares no code, header or constant table with the CUDA path.
 *
 * The paper builds its method inside an existing 3DGS renderer (Sec. 1, Sec. 2)
 * without describing it; the conventions written out here are the standard
 * 3DGS ones, fixed as definitions:
 *
 *   R      rotation of the normalised quaternion (w, x, y, z)
 *   Sigma  = R S S^T R^T,  S = diag(exp(log_scale))
 *   t      = W mu + t_c            (camera space; W, t_c world->camera)
 *   cull   t_z <= 0.2, decided on the FP32 depth key (see depth_key)
 *   J      = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]]
 *   Sigma2 = J W Sigma W^T J^T + 0.3 I,  conic Q = Sigma2^-1
 *   mean2  = (fx tx/tz + cx, fy ty/tz + cy);  pixel (u, v) samples (u+.5, v+.5)
 *   colour = max(0, sum_k sh[k] Y_k(dir) + 0.5), dir = normalise(mu - cam centre)
 *   alpha  = min(0.99, sigmoid(o) exp(-1/2 d^T Q d)); skipped if alpha < 1/255;
 *            compositing stops before the Gaussian whose T (1 - alpha) < 1e-4
 *   order  ascending depth key, equal keys by ascending index
 *   C      = sum_i c_i alpha_i T_i (background 0)
 *   score  s_i += sum_p alpha_i(p) T_i(p) E(p)       (edge score, Sec. 1 "Edge-Score")
 *
 * Y_k are the real spherical harmonics up to degree 3 in the usual ordering
 * k = l^2 + l + m, written as Cartesian polynomials of the unit direction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16
#define ORC_PROJ_STRIDE 24

/* Layout of one projected record (doubles). */
enum {
    P_VALID = 0, P_ZKEY, P_Z, P_MX, P_MY,
    P_COV_A, P_COV_B, P_COV_C,      /* Sigma2 = [[a, b], [b, c]] */
    P_CON_A, P_CON_B, P_CON_C,      /* Q = [[A, B], [B, C]] */
    P_OPAC, P_R, P_G, P_B,
    P_RAW_R, P_RAW_G, P_RAW_B,      /* colour before the clamp at 0 */
    P_RADIUS, P_TX0, P_TY0, P_TX1, P_TY1, P_SPARE
};

typedef struct {
    const float *viewmat;  /* 12 floats: 3x4 row-major [W | t_c] */
    double fx, fy, cx, cy;
    int width, height;
} ocam;

/* ---------------------------------------------------------------- helpers */

/* Depth key in FP32 with an explicit fma order.  The depth order and the
 * near-plane cull are decisions, so the oracle takes them in the same
 * precision as the device (both sides evaluate this exact expression). */
static float depth_key(const float *vm, const float *mu)
{
    return fmaf(vm[8], mu[0], fmaf(vm[9], mu[1], fmaf(vm[10], mu[2], vm[11])));
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static void quat_to_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR/dq for the normalised quaternion: dR[e][j] = d R_e / d q_j. */
static void quat_to_rot_jac(const double q[4], double dR[9][4])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double t[9][4] = {
        {0, 0, -4 * y, -4 * z},   {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x},
        {2 * z, 2 * y, 2 * x, 2 * w}, {0, -4 * x, 0, -4 * z},     {-2 * x, -2 * w, 2 * z, 2 * y},
        {-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y}, {0, -4 * x, -4 * y, 0}};
    memcpy(dR, t, sizeof(t));
}

/* Real spherical harmonics up to degree 3 at unit direction (x, y, z). */
static void sh_basis(double x, double y, double z, double Y[16])
{
    const double c0 = 0.28209479177387814;                 /* 1/(2 sqrt(pi)) */
    const double c1 = 0.4886025119029199;                  /* sqrt(3/(4 pi)) */
    const double c2a = 1.0925484305920792;                 /* 1/2 sqrt(15/pi) */
    const double c2b = 0.31539156525252005;                /* 1/4 sqrt(5/pi) */
    const double c2c = 0.5462742152960396;                 /* 1/4 sqrt(15/pi) */
    const double c3a = 0.5900435899266435;                 /* 1/4 sqrt(35/(2 pi)) */
    const double c3b = 2.890611442640554;                  /* 1/2 sqrt(105/pi) */
    const double c3c = 0.4570457994644658;                 /* 1/4 sqrt(21/(2 pi)) */
    const double c3d = 0.3731763325901154;                 /* 1/4 sqrt(7/pi) */
    const double c3e = 1.445305721320277;                  /* 1/4 sqrt(105/pi) */
    Y[0] = c0;
    Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
    Y[4] = c2a * x * y; Y[5] = c2a * y * z; Y[6] = c2b * (3 * z * z - 1);
    Y[7] = c2a * x * z; Y[8] = c2c * (x * x - y * y);
    Y[9] = c3a * y * (3 * x * x - y * y); Y[10] = c3b * x * y * z;
    Y[11] = c3c * y * (5 * z * z - 1);    Y[12] = c3d * z * (5 * z * z - 3);
    Y[13] = c3c * x * (5 * z * z - 1);    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3 * y * y);
}

/* Gradient of each basis polynomial with respect to (x, y, z). */
static void sh_basis_grad(double x, double y, double z, double dY[16][3])
{
    const double c1 = 0.4886025119029199, c2a = 1.0925484305920792, c2b = 0.31539156525252005;
    const double c2c = 0.5462742152960396, c3a = 0.5900435899266435, c3b = 2.890611442640554;
    const double c3c = 0.4570457994644658, c3d = 0.3731763325901154, c3e = 1.445305721320277;
    memset(dY, 0, sizeof(double) * 48);
    dY[1][1] = c1; dY[2][2] = c1; dY[3][0] = c1;
    dY[4][0] = c2a * y; dY[4][1] = c2a * x;
    dY[5][1] = c2a * z; dY[5][2] = c2a * y;
    dY[6][2] = c2b * 6 * z;
    dY[7][0] = c2a * z; dY[7][2] = c2a * x;
    dY[8][0] = c2c * 2 * x; dY[8][1] = -c2c * 2 * y;
    dY[9][0] = c3a * 6 * x * y; dY[9][1] = c3a * (3 * x * x - 3 * y * y);
    dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
    dY[11][1] = c3c * (5 * z * z - 1); dY[11][2] = c3c * 10 * y * z;
    dY[12][2] = c3d * (15 * z * z - 3);
    dY[13][0] = c3c * (5 * z * z - 1); dY[13][2] = c3c * 10 * x * z;
    dY[14][0] = c3e * 2 * x * z; dY[14][1] = -c3e * 2 * y * z; dY[14][2] = c3e * (x * x - y * y);
    dY[15][0] = c3a * (3 * x * x - 3 * y * y); dY[15][1] = -c3a * 6 * x * y;
}

static void cam_center(const float *vm, double c[3])
{
    /* c = -W^T t_c */
    for (int j = 0; j < 3; j++)
        c[j] = -((double)vm[0 + j] * vm[3] + (double)vm[4 + j] * vm[7] + (double)vm[8 + j] * vm[11]);
}

int orc_sh_basis(int64_t n, const double *dirs, double *out)
{
    for (int64_t i = 0; i < n; i++) sh_basis(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], out + 16 * i);
    return 0;
}

int orc_quat_to_rot(int64_t n, const double *q, double *out)
{
    for (int64_t i = 0; i < n; i++) {
        double nq = sqrt(q[4 * i] * q[4 * i] + q[4 * i + 1] * q[4 * i + 1] + q[4 * i + 2] * q[4 * i + 2] +
                         q[4 * i + 3] * q[4 * i + 3]);
        double qn[4] = {q[4 * i] / nq, q[4 * i + 1] / nq, q[4 * i + 2] / nq, q[4 * i + 3] / nq};
        quat_to_rot(qn, out + 9 * i);
    }
    return 0;
}

/* ------------------------------------------------------------- projection */

static void project_one(int64_t i, const double *means, const double *log_scales, const double *quats,
                        const double *opac_logits, const double *sh, int sh_degree, const ocam *cam,
                        double *rec)
{
    const float *vm = cam->viewmat;
    const float mu32[3] = {(float)means[3 * i], (float)means[3 * i + 1], (float)means[3 * i + 2]};
    int K = (sh_degree + 1) * (sh_degree + 1);
    memset(rec, 0, sizeof(double) * ORC_PROJ_STRIDE);
    float zkey = depth_key(vm, mu32);
    rec[P_ZKEY] = zkey;
    if (!(zkey > 0.2f)) return;

    double mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    double W[9];
    for (int e = 0; e < 3; e++)
        for (int j = 0; j < 3; j++) W[3 * e + j] = vm[4 * e + j];
    double t[3];
    for (int e = 0; e < 3; e++) t[e] = W[3 * e] * mu[0] + W[3 * e + 1] * mu[1] + W[3 * e + 2] * mu[2] + vm[4 * e + 3];

    double q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int j = 0; j < 4; j++) q[j] /= nq;
    double R[9];
    quat_to_rot(q, R);
    double s[3] = {exp(log_scales[3 * i]), exp(log_scales[3 * i + 1]),
                   exp(log_scales[3 * i + 2])};
    double Sig[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += R[3 * a + k] * s[k] * s[k] * R[3 * b + k];
            Sig[3 * a + b] = acc;
        }
    double tz = t[2];
    double J[6] = {cam->fx / tz, 0, -cam->fx * t[0] / (tz * tz), 0, cam->fy / tz, -cam->fy * t[1] / (tz * tz)};
    double T[6]; /* T = J W */
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 3; b++) T[3 * a + b] = J[3 * a] * W[b] + J[3 * a + 1] * W[3 + b] + J[3 * a + 2] * W[6 + b];
    double S2[4];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            double acc = 0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) acc += T[3 * a + k] * Sig[3 * k + l] * T[3 * b + l];
            S2[2 * a + b] = acc;
        }
    double ca = S2[0] + 0.3, cb = S2[1], cc = S2[3] + 0.3;
    double det = ca * cc - cb * cb;
    if (!(det > 0)) return;
    double opac = sigmoid(opac_logits[i]);

    double cc3[3];
    cam_center(vm, cc3);
    double d[3] = {mu[0] - cc3[0], mu[1] - cc3[1], mu[2] - cc3[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Y[16];
    sh_basis(d[0] / dn, d[1] / dn, d[2] / dn, Y);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.5;
        for (int k = 0; k < K; k++) acc += sh[(i * K + k) * 3 + ch] * Y[k];
        rec[P_RAW_R + ch] = acc;
        rec[P_R + ch] = acc > 0 ? acc : 0;
    }
    rec[P_VALID] = 1;
    rec[P_Z] = tz;
    rec[P_MX] = cam->fx * t[0] / tz + cam->cx;
    rec[P_MY] = cam->fy * t[1] / tz + cam->cy;
    rec[P_COV_A] = ca; rec[P_COV_B] = cb; rec[P_COV_C] = cc;
    rec[P_CON_A] = cc / det; rec[P_CON_B] = -cb / det; rec[P_CON_C] = ca / det;
    rec[P_OPAC] = opac;
    /* Footprint used only to bin pixels into tiles: every pixel whose alpha
     * can reach 1/255 lies within radius sqrt(2 ln(255 o) lambda_max) of the
     * mean, since d^T Q d >= |d|^2 / lambda_max. */
    double radius = -1;
    if (opac * 255.0 > 1.0) {
        double mid = 0.5 * (ca + cc);
        double lmax = mid + sqrt(mid * mid - det > 0 ? mid * mid - det : 0);
        radius = sqrt(2.0 * log(255.0 * opac) * lmax);
    }
    rec[P_RADIUS] = radius;
    if (radius >= 0) {
        rec[P_TX0] = floor((rec[P_MX] - radius - 0.5) / ORC_TILE);
        rec[P_TY0] = floor((rec[P_MY] - radius - 0.5) / ORC_TILE);
        rec[P_TX1] = floor((rec[P_MX] + radius - 0.5) / ORC_TILE);
        rec[P_TY1] = floor((rec[P_MY] + radius - 0.5) / ORC_TILE);
    }
}

int orc_project(int64_t n, const double *means, const double *log_scales, const double *quats,
                const double *opac_logits, const double *sh, int sh_degree, const float *viewmat,
                const double *intr, int width, int height, double *out)
{
    ocam cam = {viewmat, intr[0], intr[1], intr[2], intr[3], width, height};
    for (int64_t i = 0; i < n; i++)
        project_one(i, means, log_scales, quats, opac_logits, sh, sh_degree, &cam, out + i * ORC_PROJ_STRIDE);
    return 0;
}

/* ---------------------------------------------------------- compositing */

typedef struct { float key; int64_t id; } okey;

static int cmp_key(const void *a, const void *b)
{
    const okey *x = a, *y = b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Valid Gaussians in compositing order. */
static int64_t sorted_order(int64_t n, const double *proj, int64_t *order)
{
    okey *k = malloc(sizeof(okey) * (n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (proj[i * ORC_PROJ_STRIDE + P_VALID] != 0) {
            k[m].key = (float)proj[i * ORC_PROJ_STRIDE + P_ZKEY];
            k[m].id = i;
            m++;
        }
    qsort(k, m, sizeof(okey), cmp_key);
    for (int64_t j = 0; j < m; j++) order[j] = k[j].id;
    free(k);
    return m;
}

/* Per-tile lists (CSR) of the Gaussians whose footprint square meets the
 * tile, each list in compositing order. */
typedef struct { int tx, ty; int64_t *start; int64_t *ids; } otiles;

static void build_tiles(int64_t m, const int64_t *order, const double *proj, int width, int height,
                        const int *pix_region, otiles *tl)
{
    int tx = (width + ORC_TILE - 1) / ORC_TILE, ty = (height + ORC_TILE - 1) / ORC_TILE;
    int64_t nt = (int64_t)tx * ty;
    /* only the tiles that hold pixels of the region get lists */
    int rx0 = 0, ry0 = 0, rx1 = tx - 1, ry1 = ty - 1;
    if (pix_region) {
        rx0 = pix_region[0] / ORC_TILE; ry0 = pix_region[1] / ORC_TILE;
        rx1 = (pix_region[2] - 1) / ORC_TILE; ry1 = (pix_region[3] - 1) / ORC_TILE;
    }
    int64_t *cnt = calloc(nt + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t j = 0; j < m; j++) {
            const double *r = proj + order[j] * ORC_PROJ_STRIDE;
            if (r[P_RADIUS] < 0) continue;
            int x0 = (int)fmax(r[P_TX0], rx0), y0 = (int)fmax(r[P_TY0], ry0);
            int x1 = (int)fmin(r[P_TX1], rx1), y1 = (int)fmin(r[P_TY1], ry1);
            for (int yy = y0; yy <= y1; yy++)
                for (int xx = x0; xx <= x1; xx++) {
                    int64_t t = (int64_t)yy * tx + xx;
                    if (pass == 0) cnt[t + 1]++;
                    else tl->ids[cnt[t]++] = order[j];
                }
        }
        if (pass == 0) {
            for (int64_t t = 0; t < nt; t++) cnt[t + 1] += cnt[t];
            tl->start = malloc(sizeof(int64_t) * (nt + 1));
            memcpy(tl->start, cnt, sizeof(int64_t) * (nt + 1));
            tl->ids = malloc(sizeof(int64_t) * (cnt[nt] > 0 ? cnt[nt] : 1));
        }
    }
    tl->tx = tx;
    tl->ty = ty;
    free(cnt);
}

typedef struct {
    int64_t id;
    double alpha, T, G, raw; /* raw = o G before the 0.99 clamp */
} ocontrib;

static double rel_gap(double a, double b) { return fabs(a - b) / fmax(fabs(a), fabs(b)); }

/* Composite one pixel over the candidate list; returns the contributors. */
static int composite_pixel(const int64_t *cand, int64_t nc, const double *proj, double px, double py,
                           ocontrib *out, double *T_final, double *gate_gap)
{
    double T = 1.0, gap = INFINITY;
    int n = 0;
    for (int64_t j = 0; j < nc; j++) {
        const double *r = proj + cand[j] * ORC_PROJ_STRIDE;
        double dx = px - r[P_MX], dy = py - r[P_MY];
        double power = -0.5 * (r[P_CON_A] * dx * dx + 2.0 * r[P_CON_B] * dx * dy + r[P_CON_C] * dy * dy);
        double G = exp(power);
        double raw = r[P_OPAC] * G;
        double alpha = raw < 0.99 ? raw : 0.99;
        gap = fmin(gap, rel_gap(alpha, 1.0 / 255.0));
        if (alpha < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - alpha);
        gap = fmin(gap, rel_gap(Tn, 1e-4));
        if (Tn < 1e-4) break;
        out[n].id = cand[j];
        out[n].alpha = alpha;
        out[n].T = T;
        out[n].G = G;
        out[n].raw = raw;
        n++;
        T = Tn;
    }
    *T_final = T;
    if (gate_gap) *gate_gap = gap;
    return n;
}

/* The valid Gaussians in compositing order (returns their number). */
int64_t orc_order(int64_t n, const double *proj, int64_t *order) { return sorted_order(n, proj, order); }

/* Mark (mark[id] = 1) the Gaussians whose result at one of the npx listed
 * pixels (xy = x0, y0, x1, y1, ...) moves when one gate decision at that pixel
 * goes the other way: every Gaussian composited there, every candidate whose
 * alpha lies within `window` relative of 1/255 (or whose unclamped alpha lies
 * that close to the 0.99 clamp), the one at which compositing stops and the
 * next candidate past it that passes the alpha gate.  order holds
 * the m valid Gaussians in compositing order; candidates are the tile-list
 * members of the pixel's tile, as in orc_render.  Used to exempt Gaussians
 * from parity checks next to gates decided in different precisions. */
int orc_gate_affected(int64_t m, const int64_t *order, const double *proj, int64_t npx, const int32_t *xy,
                      double window, uint8_t *mark)
{
    /* tile rectangles in compositing order, contiguous */
    int32_t *rect = malloc(sizeof(int32_t) * 4 * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; j++) {
        const double *r = proj + order[j] * ORC_PROJ_STRIDE;
        int32_t *q = rect + 4 * j;
        if (r[P_RADIUS] < 0) { q[0] = 1; q[2] = 0; q[1] = 1; q[3] = 0; continue; }
        q[0] = (int32_t)r[P_TX0]; q[1] = (int32_t)r[P_TY0]; q[2] = (int32_t)r[P_TX1]; q[3] = (int32_t)r[P_TY1];
    }
    for (int64_t p = 0; p < npx; p++) {
        int x = xy[2 * p], y = xy[2 * p + 1];
        int tx = x / ORC_TILE, ty = y / ORC_TILE;
        double px = x + 0.5, py = y + 0.5, T = 1.0;
        int stopped = 0;
        for (int64_t j = 0; j < m; j++) {
            const int32_t *q = rect + 4 * j;
            if (tx < q[0] || tx > q[2] || ty < q[1] || ty > q[3]) continue;
            const double *r = proj + order[j] * ORC_PROJ_STRIDE;
            double dx = px - r[P_MX], dy = py - r[P_MY];
            double power = -0.5 * (r[P_CON_A] * dx * dx + 2.0 * r[P_CON_B] * dx * dy + r[P_CON_C] * dy * dy);
            double raw = r[P_OPAC] * exp(power);
            double alpha = raw < 0.99 ? raw : 0.99;
            if (rel_gap(alpha, 1.0 / 255.0) < window) mark[order[j]] = 1;
            if (alpha < 1.0 / 255.0) continue;
            /* the alpha clamp at 0.99 switches the geometry gradient on and off */
            if (rel_gap(raw, 0.99) < window) mark[order[j]] = 1;
            mark[order[j]] = 1;
            if (stopped) break;
            double Tn = T * (1.0 - alpha);
            if (Tn < 1e-4) stopped = 1;
            T = Tn;
        }
    }
    free(rect);
    return 0;
}

/* Render the pixel region [x0,x1) x [y0,y1).  brute = 1 composites every
 * valid Gaussian at every pixel (no tiles, no footprint test). */
int orc_render(int64_t n, const double *proj, int width, int height, const double *edge, int brute,
               int x0, int y0, int x1, int y1, double *rgb, double *T_out, int32_t *ncontrib,
               int64_t *last_id, double *score, double *gate_gap, const int64_t *given_order, int64_t given_m)
{
    /* given_order (nullable): the valid Gaussians already in compositing order */
    int64_t *order = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t m;
    if (given_order) {
        m = given_m;
        memcpy(order, given_order, sizeof(int64_t) * (size_t)m);
    } else {
        m = sorted_order(n, proj, order);
    }
    otiles tl = {0};
    int reg[4] = {x0, y0, x1, y1};
    if (!brute) build_tiles(m, order, proj, width, height, reg, &tl);
    ocontrib *cb = malloc(sizeof(ocontrib) * (m > 0 ? m : 1));
    for (int y = y0; y < y1; y++)
        for (int x = x0; x < x1; x++) {
            const int64_t *cand = order;
            int64_t nc = m;
            if (!brute) {
                int64_t t = (int64_t)(y / ORC_TILE) * tl.tx + x / ORC_TILE;
                cand = tl.ids + tl.start[t];
                nc = tl.start[t + 1] - tl.start[t];
            }
            double T, gap;
            int nk = composite_pixel(cand, nc, proj, x + 0.5, y + 0.5, cb, &T, &gap);
            int64_t p = (int64_t)y * width + x;
            double c[3] = {0, 0, 0};
            for (int k = 0; k < nk; k++) {
                const double *r = proj + cb[k].id * ORC_PROJ_STRIDE;
                double w = cb[k].alpha * cb[k].T;
                for (int ch = 0; ch < 3; ch++) c[ch] += r[P_R + ch] * w;
                if (score && edge) score[cb[k].id] += w * edge[p];
            }
            if (rgb) for (int ch = 0; ch < 3; ch++) rgb[3 * p + ch] = c[ch];
            if (T_out) T_out[p] = T;
            if (ncontrib) ncontrib[p] = nk;
            if (last_id) last_id[p] = nk ? cb[nk - 1].id : -1;
            if (gate_gap) gate_gap[p] = gap;
        }
    free(cb);
    if (!brute) { free(tl.start); free(tl.ids); }
    free(order);
    return 0;
}

/* ------------------------------------------------------------- adjoint */

/* Gradients of L given dL/dC (H*W*3).  g2d (n x 9, nullable) receives the
 * screen-space gradients (mean2 x, y, conic A, B, C, opacity, r, g, b); the
 * parameter gradients are written (not accumulated) to the g_* arrays. */
int orc_render_bwd(int64_t n, const double *means, const double *log_scales, const double *quats,
                   const double *opac_logits, const double *sh, int sh_degree, const float *viewmat,
                   const double *intr, int width, int height, const double *proj, const double *dLdC,
                   double *g_means, double *g_log_scales, double *g_quats, double *g_opac, double *g_sh,
                   double *g2d_out, const int *region, int mag)
{
    /* mag != 0: the magnitude adjoint.  Every factor of every term enters by its
     * absolute value and every difference becomes a sum, so each output is the
     * sum of the absolute values of the terms that the plain adjoint adds up: the
     * condition of that sum, which bounds how far relative perturbations of the
     * terms (rounding in a lower precision) can move the result.  mag == 0
     * evaluates exactly the plain adjoint. */
#define MG(x) (mag ? fabs(x) : (x))
#define DIFF(a, b) (mag ? fabs(a) + fabs(b) : (a) - (b))
    /* region (nullable): only pixels of [x0,x1) x [y0,y1) carry dL/dC (the others are taken as 0) */
    int rx0 = 0, ry0 = 0, rx1 = width, ry1 = height;
    if (region) { rx0 = region[0]; ry0 = region[1]; rx1 = region[2]; ry1 = region[3]; }
    int K = (sh_degree + 1) * (sh_degree + 1);
    (void)opac_logits; /* sigmoid(o) is read from the projected record */
    double *g2d = calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
    int64_t *order = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t m = sorted_order(n, proj, order);
    otiles tl = {0};
    build_tiles(m, order, proj, width, height, region, &tl);
    ocontrib *cb = malloc(sizeof(ocontrib) * (m > 0 ? m : 1));

    for (int y = ry0; y < ry1; y++)
        for (int x = rx0; x < rx1; x++) {
            int64_t t = (int64_t)(y / ORC_TILE) * tl.tx + x / ORC_TILE;
            double T;
            int nk = composite_pixel(tl.ids + tl.start[t], tl.start[t + 1] - tl.start[t], proj, x + 0.5,
                                     y + 0.5, cb, &T, NULL);
            const double *g = dLdC + 3 * ((int64_t)y * width + x);
            for (int k = 0; k < nk; k++) {
                const double *r = proj + cb[k].id * ORC_PROJ_STRIDE;
                double *o = g2d + 9 * cb[k].id;
                /* dC/dc_k = alpha_k T_k */
                for (int ch = 0; ch < 3; ch++) o[6 + ch] += MG(g[ch]) * cb[k].alpha * cb[k].T;
                /* dC/dalpha_k = T_k c_k - sum_{j>k} c_j alpha_j T_j / (1 - alpha_k) */
                double dalpha = 0;
                for (int ch = 0; ch < 3; ch++) {
                    double behind = 0;
                    for (int j = k + 1; j < nk; j++)
                        behind += proj[cb[j].id * ORC_PROJ_STRIDE + P_R + ch] * cb[j].alpha * cb[j].T;
                    dalpha += MG(g[ch]) * DIFF(cb[k].T * r[P_R + ch], behind / (1.0 - cb[k].alpha));
                }
                if (cb[k].raw >= 0.99) continue; /* clamped alpha: constant */
                double G = cb[k].G;
                double dx = x + 0.5 - r[P_MX], dy = y + 0.5 - r[P_MY];
                o[5] += dalpha * G;
                double dG = dalpha * r[P_OPAC];
                o[0] += dG * G * (MG(r[P_CON_A] * dx) + MG(r[P_CON_B] * dy));
                o[1] += dG * G * (MG(r[P_CON_B] * dx) + MG(r[P_CON_C] * dy));
                o[2] += dG * G * MG(-0.5 * dx * dx);
                o[3] += dG * G * MG(-dx * dy);
                o[4] += dG * G * MG(-0.5 * dy * dy);
            }
        }
    free(cb);
    free(tl.start);
    free(tl.ids);
    free(order);

    const float *vm = viewmat;
    double W[9];
    for (int e = 0; e < 3; e++)
        for (int j = 0; j < 3; j++) W[3 * e + j] = vm[4 * e + j];
    double ccen[3];
    cam_center(vm, ccen);
    double fx = intr[0], fy = intr[1];

    for (int64_t i = 0; i < n; i++) {
        const double *r = proj + i * ORC_PROJ_STRIDE;
        double *o = g2d + 9 * i;
        for (int j = 0; j < 3; j++) g_means[3 * i + j] = 0, g_log_scales[3 * i + j] = 0;
        for (int j = 0; j < 4; j++) g_quats[4 * i + j] = 0;
        g_opac[i] = 0;
        for (int j = 0; j < 3 * K; j++) g_sh[3 * K * i + j] = 0;
        if (r[P_VALID] == 0) continue;

        double mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
        double t[3];
        for (int e = 0; e < 3; e++) t[e] = W[3 * e] * mu[0] + W[3 * e + 1] * mu[1] + W[3 * e + 2] * mu[2] + vm[4 * e + 3];
        double tz = t[2];
        double q0[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
        double nq = sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
        double q[4] = {q0[0] / nq, q0[1] / nq, q0[2] / nq, q0[3] / nq};
        double R[9];
        quat_to_rot(q, R);
        double s[3] = {exp(log_scales[3 * i]), exp(log_scales[3 * i + 1]),
                       exp(log_scales[3 * i + 2])};
        double Mm[9]; /* M = R S */
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) Mm[3 * a + b] = R[3 * a + b] * s[b];
        double Sig[9];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0;
                for (int k = 0; k < 3; k++) acc += Mm[3 * a + k] * Mm[3 * b + k];
                Sig[3 * a + b] = acc;
            }
        double J[6] = {fx / tz, 0, -fx * t[0] / (tz * tz), 0, fy / tz, -fy * t[1] / (tz * tz)};
        double T[6];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 3; b++) T[3 * a + b] = J[3 * a] * W[b] + J[3 * a + 1] * W[3 + b] + J[3 * a + 2] * W[6 + b];

        /* conic -> Sigma2:  dL/dSigma2 = -Q G_Q Q, G_Q the symmetric gradient */
        double Q[4] = {r[P_CON_A], r[P_CON_B], r[P_CON_B], r[P_CON_C]};
        double GQ[4] = {o[2], 0.5 * o[3], 0.5 * o[3], o[4]};
        double tmp[4], GS2[4];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) tmp[2 * a + b] = MG(Q[2 * a] * GQ[b]) + MG(Q[2 * a + 1] * GQ[2 + b]);
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) GS2[2 * a + b] = MG(-tmp[2 * a] * Q[b]) + MG(-tmp[2 * a + 1] * Q[2 + b]);

        /* Sigma2 = T Sigma T^T + 0.3 I */
        double GSig[9], GT[6];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0;
                for (int k = 0; k < 2; k++)
                    for (int l = 0; l < 2; l++) acc += MG(T[3 * k + a] * GS2[2 * k + l] * T[3 * l + b]);
                GSig[3 * a + b] = acc;
            }
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0;
                for (int l = 0; l < 2; l++)
                    for (int k = 0; k < 3; k++) acc += MG(GS2[2 * a + l] * T[3 * l + k] * Sig[3 * k + b]);
                GT[3 * a + b] = 2.0 * acc;
            }
        /* T = J W  ->  dL/dJ = GT W^T */
        double GJ[6];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 3; b++)
                GJ[3 * a + b] = MG(GT[3 * a] * W[3 * b]) + MG(GT[3 * a + 1] * W[3 * b + 1]) + MG(GT[3 * a + 2] * W[3 * b + 2]);
        double gt[3] = {0, 0, 0};
        /* J entries */
        gt[2] += MG(GJ[0] * (-fx / (tz * tz)));
        gt[0] += MG(GJ[2] * (-fx / (tz * tz)));
        gt[2] += MG(GJ[2] * (2.0 * fx * t[0] / (tz * tz * tz)));
        gt[2] += MG(GJ[4] * (-fy / (tz * tz)));
        gt[1] += MG(GJ[5] * (-fy / (tz * tz)));
        gt[2] += MG(GJ[5] * (2.0 * fy * t[1] / (tz * tz * tz)));
        /* mean2 */
        gt[0] += MG(o[0] * fx / tz);
        gt[2] += MG(o[0] * (-fx * t[0] / (tz * tz)));
        gt[1] += MG(o[1] * fy / tz);
        gt[2] += MG(o[1] * (-fy * t[1] / (tz * tz)));
        for (int j = 0; j < 3; j++) g_means[3 * i + j] = MG(W[j] * gt[0]) + MG(W[3 + j] * gt[1]) + MG(W[6 + j] * gt[2]);

        /* Sigma = M M^T: dL/dM = 2 GSig M (GSig symmetric) */
        double GM[9];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0;
                for (int k = 0; k < 3; k++) acc += MG((GSig[3 * a + k] + GSig[3 * k + a]) * Mm[3 * k + b]);
                GM[3 * a + b] = acc;
            }
        for (int b = 0; b < 3; b++) {
            double gs = 0;
            for (int a = 0; a < 3; a++) gs += MG(GM[3 * a + b] * R[3 * a + b]);
            g_log_scales[3 * i + b] = gs * s[b];
        }
        double GR[9];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) GR[3 * a + b] = GM[3 * a + b] * s[b];
        double dR[9][4];
        quat_to_rot_jac(q, dR);
        double gqn[4] = {0, 0, 0, 0};
        for (int e = 0; e < 9; e++)
            for (int j = 0; j < 4; j++) gqn[j] += MG(GR[e] * dR[e][j]);
        double dotq = MG(gqn[0] * q[0]) + MG(gqn[1] * q[1]) + MG(gqn[2] * q[2]) + MG(gqn[3] * q[3]);
        for (int j = 0; j < 4; j++) g_quats[4 * i + j] = DIFF(gqn[j], q[j] * dotq) / nq;

        g_opac[i] = o[5] * r[P_OPAC] * (1.0 - r[P_OPAC]);

        /* colour */
        double d[3] = {mu[0] - ccen[0], mu[1] - ccen[1], mu[2] - ccen[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double u[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
        double Y[16], dY[16][3];
        sh_basis(u[0], u[1], u[2], Y);
        sh_basis_grad(u[0], u[1], u[2], dY);
        double gu[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ch++) {
            if (r[P_RAW_R + ch] < 0) continue;
            double gc = o[6 + ch];
            for (int k = 0; k < K; k++) {
                g_sh[(i * K + k) * 3 + ch] = MG(gc * Y[k]);
                for (int a = 0; a < 3; a++) gu[a] += MG(gc * sh[(i * K + k) * 3 + ch] * dY[k][a]);
            }
        }
        double udot = MG(gu[0] * u[0]) + MG(gu[1] * u[1]) + MG(gu[2] * u[2]);
        for (int a = 0; a < 3; a++) g_means[3 * i + a] += DIFF(gu[a], u[a] * udot) / dn;
    }
    if (g2d_out) memcpy(g2d_out, g2d, sizeof(double) * 9 * n);
    free(g2d);
    return 0;
#undef MG
#undef DIFF
}
