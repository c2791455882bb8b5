// Tile-binned Gaussian splatting with per-Gaussian edge score, and its adjoint.
//
// The paper builds on an existing 3DGS renderer without describing it (Sec. 1,
// Sec. 2); the conventions implemented here are listed in gsp.h.  The edge
// score s_i = sum_p alpha_i(p) T_i(p) E(p) is the per-Gaussian importance the
// densification selects on (Sec. 1, "Edge-Score importance").
//
// Pipeline of gsp_render_fwd (all asynchronous on the caller's stream):
//   project   one thread per Gaussian reads its parameters once and projects
//             them into every view: screen mean, conic, opacity, SH colour,
//             FP32 depth key and the tile rectangle of its 1/255 footprint
//   sort      per view, stable LSD radix sort of the depth keys (4 x 8 bits),
//             ties keep ascending index
//   bin       per view, the depth-ordered Gaussians are cut into chunks;
//             per-chunk tile counts, a scan over chunks per tile and over
//             tiles give every (tile, chunk) its output range, and a stable
//             scatter writes each tile's list already in depth order (no sort
//             over the pairs)
//   composite one 256-thread block per 16x16 tile, Gaussians staged through
//             shared memory in batches, block-wide early exit
// gsp_render_bwd replays each pixel back to front from T_final and the
// last-contributor position, reduces the per-Gaussian screen-space gradients
// over the block (warp transpose-reduction, shared-memory accumulation, one
// global atomic per Gaussian, tile and value) and then chains them to the
// parameters, one thread per Gaussian over all views.
#include <algorithm>

#include "common.cuh"

namespace gsp {
namespace {

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2E = 1.4426950408889634f;  // log2(e): the stored conic gives power in base 2
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kNear = 0.2f;
constexpr int kRowCap = 16;  // tile rows per Gaussian with an exact column interval
constexpr int kProjBwdThreads = 128;

struct ViewP {
    float vm[12];
    float fx, fy, cx, cy;
    float ccx, ccy, ccz;  // camera centre in world space
    int w, h;
    int tiles_x, tiles_y;
    int tile_base;        // first global tile of the view
    int sx, sy;           // supertiles per row / column
    int super_base;       // first global supertile of the view
    long long pix_off;    // first pixel of the view
    const uint8_t *tgt;   // target image (or null)
    long long tgt_pitch;
};

struct Views {
    ViewP v[GSP_MAX_VIEWS];
    int n;
    int total_tiles;
    int total_super;
    int smax;             // largest supertile count of a view
    long long total_pix;
};

struct Params {
    const float *means, *log_scales, *quats, *opac, *sh;
    const int32_t *count;
    long long cap;
    int K;  // SH coefficients per channel
    int32_t *status = nullptr;  // device status word (bounded waits report here)
    bool sh_bulk = false;       // sh is 16-byte aligned: the projection streams it by bulk copies
    long long sh_wait_limit = kDefaultSpinLimit;  // polls of a thread's wait for the SH copy (0: gives up at once)
};

struct State {
    float4 *xyo;   // [V][cap] (mean x, mean y, opacity, bbox half-width)
    float2 *mlo;   // [V][cap] residual of the projected mean: mean = xyo.xy + mlo (double-float)
    float4 *con;   // [V][cap] log2(e) (-A/2, -B, -C/2) of the conic Q = [[A, B], [B, C]], bbox half-height
    float4 *col;   // [V][cap] (r, g, b, clamp bits)
    uint2 *rect;   // [V][cap] (tx0 | ty0 << 16, tx1 | ty1 << 16); empty if tx1 < tx0
    uchar2 *rowint;  // [V][cap][kRowCap] per tile row of the rectangle: columns (lo, hi) - tx0 the
                     // 1/255 ellipse reaches (lo > hi: none); rows past kRowCap are not culled
    uint32_t *key, *key_alt;  // depth keys [V][cap], sort scratch [V][cap]
    int32_t *val, *val_alt;   // depth-ordered ids [V][cap], sort scratch [V][cap]
    unsigned *sort_state;     // [V][4][nb_max][256] look-back words of the depth sort
    unsigned *sort_ghist;     // [V][4][256] digit counts of the four passes
    unsigned *sort_ticket;    // [V][4] tile tickets of the four passes
    unsigned *scan_ticket;    // [2] blocks done in l1_scan, l2_scan (the last one scans the totals)
    unsigned *count1;         // [total_super][nch1_max] level-1 chunk counts, then offsets
    unsigned *len1;           // [total_super] supertile list lengths
    unsigned *list1_start;    // [total_super] supertile list starts in id1
    unsigned *chunk2_base;    // [total_super + 1] first level-2 chunk of each supertile
    int32_t *id1;             // [pair_cap] supertile lists of Gaussian ids
    unsigned long long *mask1;  // [pair_cap] tile mask of each supertile entry
    unsigned *count2;         // [chunk2_cap][64] level-2 chunk counts, then offsets
    int32_t *chunk_super;     // [chunk2_cap] supertile of each level-2 chunk
    unsigned *tile_len;       // [total_tiles] list length of each tile
    unsigned *tile_start;     // [total_tiles] first position of each tile's list in ids
    unsigned *tile_avail;     // [total_tiles] entries of each tile's list written to ids (a prefix)
    unsigned *tile_redo;      // [total_tiles] 1: the tile needed more than its prefix (forward)
    unsigned *super_redo;     // [total_super] 1: a tile of the supertile needed more than its prefix
    unsigned *redo_count;     // [1] tiles in redo_list
    int32_t *redo_list;       // [total_tiles] tiles whose compositing resumes past their prefix
    int32_t *ids;             // [pair_cap] Gaussian ids, tile lists one after another
    int32_t *order_fwd;       // [total_tiles] tiles by descending list length
    int32_t *order_bwd;       // [total_tiles] tiles by descending last contributor
    unsigned *tile_work;      // [total_tiles] largest last-contributor position of each tile
    long long *contrib;       // [1] composited (pixel, Gaussian) pairs of the forward pass
    long long *pairs_total;   // [1] tile-Gaussian pairs (exact, also when over capacity)
    float4 *g2d;              // [V][cap][3]
    double *loss_acc;         // [1]
    int32_t *overflow;        // [1]
    int32_t *status = nullptr;  // the caller's device status word (bounds-checked build)
    const int32_t *n_dev;     // the caller's device count of live Gaussians
    int nb_max;               // depth-sort blocks for cap
    int nch1_max;             // level-1 chunks for cap
    unsigned prefix = 0xffffffffu;  // tile-list entries written before the forward compositing
    long long pair_cap;
};

__device__ __forceinline__ int find_view(const Views &vs, int gt)
{
    int v = 0;
    while (v + 1 < vs.n && vs.v[v + 1].tile_base <= gt) ++v;
    return v;
}

// ------------------------------------------------------------ SH basis (FP32)

constexpr float C0 = 0.28209479177387814f;
constexpr float C1 = 0.4886025119029199f;
constexpr float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
constexpr float C3a = 0.5900435899266435f, C3b = 2.890611442640554f, C3c = 0.4570457994644658f;
constexpr float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;

__device__ __forceinline__ void sh_eval(float x, float y, float z, int K, float Y[16])
{
    Y[0] = C0;
    if (K > 1) {
        Y[1] = C1 * y; Y[2] = C1 * z; Y[3] = C1 * x;
    }
    if (K > 4) {
        Y[4] = C2a * x * y; Y[5] = C2a * y * z; Y[6] = C2b * (3.f * z * z - 1.f);
        Y[7] = C2a * x * z; Y[8] = C2c * (x * x - y * y);
    }
    if (K > 9) {
        Y[9] = C3a * y * (3.f * x * x - y * y); Y[10] = C3b * x * y * z;
        Y[11] = C3c * y * (5.f * z * z - 1.f); Y[12] = C3d * z * (5.f * z * z - 3.f);
        Y[13] = C3c * x * (5.f * z * z - 1.f); Y[14] = C3e * z * (x * x - y * y);
        Y[15] = C3a * x * (x * x - 3.f * y * y);
    }
}

// sum_k w[k] * grad Y_k at (x, y, z), the basis polynomials differentiated in R^3
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, int K, const float w[16], float g[3])
{
    g[0] = g[1] = g[2] = 0.f;
    if (K > 1) {
        g[1] += C1 * w[1]; g[2] += C1 * w[2]; g[0] += C1 * w[3];
    }
    if (K > 4) {
        g[0] += C2a * y * w[4]; g[1] += C2a * x * w[4];
        g[1] += C2a * z * w[5]; g[2] += C2a * y * w[5];
        g[2] += C2b * 6.f * z * w[6];
        g[0] += C2a * z * w[7]; g[2] += C2a * x * w[7];
        g[0] += C2c * 2.f * x * w[8]; g[1] -= C2c * 2.f * y * w[8];
    }
    if (K > 9) {
        g[0] += C3a * 6.f * x * y * w[9]; g[1] += C3a * 3.f * (x * x - y * y) * w[9];
        g[0] += C3b * y * z * w[10]; g[1] += C3b * x * z * w[10]; g[2] += C3b * x * y * w[10];
        g[1] += C3c * (5.f * z * z - 1.f) * w[11]; g[2] += C3c * 10.f * y * z * w[11];
        g[2] += C3d * (15.f * z * z - 3.f) * w[12];
        g[0] += C3c * (5.f * z * z - 1.f) * w[13]; g[2] += C3c * 10.f * x * z * w[13];
        g[0] += C3e * 2.f * x * z * w[14]; g[1] -= C3e * 2.f * y * z * w[14]; g[2] += C3e * (x * x - y * y) * w[14];
        g[0] += C3a * 3.f * (x * x - y * y) * w[15]; g[1] -= C3a * 6.f * x * y * w[15];
    }
}

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Depth key: the same fma order the FP64 reference uses for this decision.
__device__ __forceinline__ float depth_key(const float *vm, float mx, float my, float mz)
{
    return __fmaf_rn(vm[8], mx, __fmaf_rn(vm[9], my, __fmaf_rn(vm[10], mz, vm[11])));
}

struct Proj {
    float tx, ty, tz;
    float R[9], s[3];
    float Sig[6];   // xx xy xz yy yz zz
    float T[6];     // J W
    float a, b, c;  // Sigma2 (with +0.3)
    float det;
};

__device__ __forceinline__ void project_geom(const ViewP &V, const float *mu, const float *ls, const float *q4,
                                             Proj &P)
{
    const float *vm = V.vm;
    P.tz = depth_key(vm, mu[0], mu[1], mu[2]);
    P.tx = vm[0] * mu[0] + vm[1] * mu[1] + vm[2] * mu[2] + vm[3];
    P.ty = vm[4] * mu[0] + vm[5] * mu[1] + vm[6] * mu[2] + vm[7];
    float qn = __frsqrt_rn(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
    quat_rot(q4[0] * qn, q4[1] * qn, q4[2] * qn, q4[3] * qn, P.R);
    P.s[0] = expf(ls[0]); P.s[1] = expf(ls[1]); P.s[2] = expf(ls[2]);
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M[3 * a + b] = P.R[3 * a + b] * P.s[b];
    P.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    P.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    P.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    P.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    P.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    P.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    float iz = 1.f / P.tz;
    float j00 = V.fx * iz, j02 = -V.fx * P.tx * iz * iz;
    float j11 = V.fy * iz, j12 = -V.fy * P.ty * iz * iz;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        P.T[b] = j00 * vm[b] + j02 * vm[8 + b];
        P.T[3 + b] = j11 * vm[4 + b] + j12 * vm[8 + b];
    }
    // Sigma2 = T Sig T^T
    const float *S = P.Sig;
    float u0 = P.T[0] * S[0] + P.T[1] * S[1] + P.T[2] * S[2];
    float u1 = P.T[0] * S[1] + P.T[1] * S[3] + P.T[2] * S[4];
    float u2 = P.T[0] * S[2] + P.T[1] * S[4] + P.T[2] * S[5];
    float v0 = P.T[3] * S[0] + P.T[4] * S[1] + P.T[5] * S[2];
    float v1 = P.T[3] * S[1] + P.T[4] * S[3] + P.T[5] * S[4];
    float v2 = P.T[3] * S[2] + P.T[4] * S[4] + P.T[5] * S[5];
    P.a = u0 * P.T[0] + u1 * P.T[1] + u2 * P.T[2] + 0.3f;
    P.b = u0 * P.T[3] + u1 * P.T[4] + u2 * P.T[5];
    P.c = v0 * P.T[3] + v1 * P.T[4] + v2 * P.T[5] + 0.3f;
    P.det = P.a * P.c - P.b * P.b;
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// --------------------------------------------------------------- projection

// The SH coefficients of one Gaussian (3K floats) into registers; 16-byte
// loads when the row length allows (K = 4, 16).
// acc[ch] += sum_k row[3k + ch] * Y[k], the coefficients streamed from memory in
// 16-byte loads (row-major [K][3]; terms added in ascending k per channel).
// SMEM: the row is in shared memory (generic loads instead of read-only global ones).
template <int K, bool SMEM = false>
__device__ __forceinline__ void sh_weighted(const float *row, const float Y[16], float acc[3])
{
    if constexpr ((3 * K) % 4 == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < 3 * K / 4; ++q) {
            const float4 v = SMEM ? r4[q] : __ldg(r4 + q);
            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[(4 * q + j) % 3] += e[j] * Y[(4 * q + j) / 3];
        }
    } else {
#pragma unroll
        for (int el = 0; el < 3 * K; ++el) acc[el % 3] += (SMEM ? row[el] : __ldg(row + el)) * Y[el / 3];
    }
}

// w[k] += sum_ch g[ch] * row[3k + ch] (ascending ch per k), streamed like sh_weighted.
template <int K>
__device__ __forceinline__ void sh_contract(const float *row, const float g[3], float w[16])
{
    if constexpr ((3 * K) % 4 == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < 3 * K / 4; ++q) {
            const float4 v = __ldg(r4 + q);
            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) w[(4 * q + j) / 3] += g[(4 * q + j) % 3] * e[j];
        }
    } else {
#pragma unroll
        for (int el = 0; el < 3 * K; ++el) w[el / 3] += g[el % 3] * __ldg(row + el);
    }
}

template <int K>
__device__ __forceinline__ void load_sh(const float *row, float *out)
{
    if constexpr ((3 * K) % 4 == 0) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < 3 * K / 4; ++q) {
            const float4 v = r4[q];
            out[4 * q] = v.x; out[4 * q + 1] = v.y; out[4 * q + 2] = v.z; out[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 3 * K; ++q) out[q] = row[q];
    }
}

// ---- double-float arithmetic for the projected mean (error-free transformations:
// Knuth's TwoSum, the FMA TwoProduct, and the compensated dot product of Ogita,
// Rump and Oishi, "Accurate sum and dot product", 2005)

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// r0 a + r1 b + r2 c + r3 as hi + lo (compensated dot product)
__device__ __forceinline__ void dot3_plus(const float *r, float a, float b, float c, float &hi, float &lo)
{
    float p0, e0, p1, e1, p2, e2, s, t;
    two_prod(r[0], a, p0, e0);
    two_prod(r[1], b, p1, e1);
    two_prod(r[2], c, p2, e2);
    two_sum(p0, p1, s, t);
    float err = __fadd_rn(__fadd_rn(e0, e1), t);
    two_sum(s, p2, s, t);
    err = __fadd_rn(err, __fadd_rn(e2, t));
    two_sum(s, r[3], s, t);
    err = __fadd_rn(err, t);
    two_sum(s, err, hi, lo);
}

// f (n / z) + c for double-float n and z, as a normalised hi + lo
__device__ __forceinline__ void df_project(float f, float c, float n_hi, float n_lo, float z_hi, float z_lo,
                                           float &hi, float &lo)
{
    const float q = __fdiv_rn(n_hi, z_hi);
    const float r = __fmaf_rn(-q, z_hi, n_hi);  // exact remainder
    const float ql = __fdiv_rn(__fadd_rn(r, __fsub_rn(n_lo, __fmul_rn(q, z_lo))), z_hi);
    float p, e, s, t;
    two_prod(f, q, p, e);
    e = __fmaf_rn(f, ql, e);
    two_sum(p, c, s, t);
    two_sum(s, __fadd_rn(e, t), hi, lo);
}

// Projected mean (fx t_x / t_z + cx, fy t_y / t_z + cy), t = W mu + t_c, to about
// 2^-44 relative: the pixel offsets of compositing then carry only their own rounding.
__device__ __forceinline__ void projected_mean(const ViewP &V, const float *mu, float &mx, float &mx_lo, float &my,
                                               float &my_lo)
{
    float xh, xl, yh, yl, zh, zl;
    dot3_plus(V.vm, mu[0], mu[1], mu[2], xh, xl);
    dot3_plus(V.vm + 4, mu[0], mu[1], mu[2], yh, yl);
    dot3_plus(V.vm + 8, mu[0], mu[1], mu[2], zh, zl);
    df_project(V.fx, V.cx, xh, xl, zh, zl, mx, mx_lo);
    df_project(V.fy, V.cy, yh, yl, zh, zl, my, my_lo);
}

// Projects Gaussian i < capacity into every view; returns its tile-Gaussian pairs.
// sh_s: the Gaussian's SH row in shared memory, valid once the bulk copy on bar
// has landed (nullptr: read it from global memory).
template <int K>
__device__ __forceinline__ unsigned long long project_one(const Views &vs, const Params &p, const State &st,
                                                          long long i, const float *sh_s,
                                                          unsigned long long *bar)
{
    bool sh_ready = false;
    const int n = *p.count;
    unsigned long long pairs = 0;
    const long long cap = p.cap;
    for (int v = 0; v < vs.n; ++v) {
        st.val[v * cap + i] = int32_t(i);
    }
    if (i >= n) return 0;
    float mu[3] = {p.means[3 * i], p.means[3 * i + 1], p.means[3 * i + 2]};
    float ls[3] = {p.log_scales[3 * i], p.log_scales[3 * i + 1], p.log_scales[3 * i + 2]};
    float q4[4] = {p.quats[4 * i], p.quats[4 * i + 1], p.quats[4 * i + 2], p.quats[4 * i + 3]};
    float opac = sigmoidf_(p.opac[i]);
    const float *shrow = p.sh + (size_t)i * K * 3;
    for (int v = 0; v < vs.n; ++v) {
        const ViewP &V = vs.v[v];
        const long long o = v * cap + i;
        Proj P;
        project_geom(V, mu, ls, q4, P);
        bool ok = P.tz > kNear && P.det > 0.f && opac >= kAlphaMin;
        uint2 rect = make_uint2(1u, 0u);  // empty
        if (ok) {
            // the projected mean as a double-float (hi + lo): an FP32 mean is off by up
            // to half an ulp of the pixel coordinate (3e-5 px at x ~ 600), which moves
            // every pixel offset d of the Gaussian by as much
            float mx, my, mx_lo, my_lo;
            projected_mean(V, mu, mx, mx_lo, my, my_lo);
            float id = 1.f / P.det;
            // footprint of alpha >= 1/255: d^T Q d <= 2 ln(255 o); its bounding box
            // has half-extents sqrt(2 ln(255 o) Sigma2_xx), sqrt(... Sigma2_yy)
            float lim = 2.f * logf(255.f * opac);
            float ex = sqrtf(fmaxf(lim, 0.f) * P.a) * 1.0001f + 0.01f;
            float ey = sqrtf(fmaxf(lim, 0.f) * P.c) * 1.0001f + 0.01f;
            int tx0 = max(int(floorf((mx - ex - 0.5f) / kTile)), 0);
            int tx1 = min(int(floorf((mx + ex - 0.5f) / kTile)), V.tiles_x - 1);
            int ty0 = max(int(floorf((my - ey - 0.5f) / kTile)), 0);
            int ty1 = min(int(floorf((my + ey - 0.5f) / kTile)), V.tiles_y - 1);
            if (tx0 <= tx1 && ty0 <= ty1) {
                rect = make_uint2(unsigned(tx0) | (unsigned(ty0) << 16), unsigned(tx1) | (unsigned(ty1) << 16));
                // exact column interval of the ellipse d^T Sigma2^-1 d <= lim over the strip of
                // pixel-centre rows of each tile row: at height dy the ellipse spans
                // x = (b/c) dy +- sqrt((lim - dy^2/c)(a - b^2/c)); the upper bound is concave in
                // dy and peaks at the rightmost point dy = b sqrt(lim/a), the lower one mirrors it
                const float la = fmaxf(lim, 0.f);
                const float ymax = sqrtf(la * P.c);
                const float dyr = P.b * sqrtf(la / P.a);
                const float inv_c = 1.f / P.c, b_c = P.b * inv_c;  // per Gaussian, not per row
                const float schur = fmaxf(P.a - P.b * b_c, 0.f);
                uchar2 *ri = st.rowint + o * kRowCap;
                const int nrows = min(ty1 - ty0 + 1, kRowCap);  // binning reads only these rows
                const int wr = tx1 - tx0 + 1;
                // rows past kRowCap, and every row of a rectangle wider than 255 tiles
                // (marked (0, 255)), keep the whole rectangle width
                pairs += (unsigned long long)(ty1 - ty0 + 1 - nrows) * wr;
                for (int yy = 0; yy < nrows && wr > 255; ++yy) {
                    ri[yy] = make_uchar2(0, 255);
                    pairs += wr;
                }
                for (int yy = 0; yy < nrows && wr <= 255; ++yy) {
                    const int ty = ty0 + yy;
                    uchar2 iv = make_uchar2(255, 0);
                    {
                        const float lo = fmaxf(float(ty * kTile) + 0.5f - my, -ymax);
                        const float hi = fminf(float(ty * kTile + kTile - 1) + 0.5f - my, ymax);
                        if (lo <= hi) {
                            const float d1 = fminf(fmaxf(dyr, lo), hi), d2 = fminf(fmaxf(-dyr, lo), hi);
                            const float xr = b_c * d1 + sqrtf(fmaxf(la - d1 * d1 * inv_c, 0.f) * schur);
                            const float xl = b_c * d2 - sqrtf(fmaxf(la - d2 * d2 * inv_c, 0.f) * schur);
                            const float m = 0.01f + 1e-4f * (fabsf(xl) + fabsf(xr));
                            const int c0 = max(int(floorf((mx + xl - m - 0.5f) / kTile)), tx0);
                            const int c1 = min(int(floorf((mx + xr + m - 0.5f) / kTile)), tx1);
                            if (c0 <= c1) {
                                iv = make_uchar2((unsigned char)(c0 - tx0), (unsigned char)(c1 - tx0));
                                pairs += c1 - c0 + 1;
                            }
                        }
                    }
                    ri[yy] = iv;
                }
            } else {
                ok = false;
            }
            // view-dependent colour
            float dx = mu[0] - V.ccx, dy = mu[1] - V.ccy, dz = mu[2] - V.ccz;
            float rn = __frsqrt_rn(dx * dx + dy * dy + dz * dz);
            float Y[16];
            sh_eval(dx * rn, dy * rn, dz * rn, K, Y);
            float col[3] = {0.5f, 0.5f, 0.5f};
            if (sh_s && !sh_ready) {
                sh_ready = mbar_wait(bar, 0, p.sh_wait_limit);
                if (!sh_ready) {
                    set_status(p.status, GSP_ERR_TIMEOUT);
                    sh_s = nullptr;  // the global row is still there
                }
            }
            if (sh_s) sh_weighted<K, true>(sh_s, Y, col);
            else sh_weighted<K>(shrow, Y, col);
            unsigned clampbits = 0;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                if (col[ch] < 0.f) {
                    clampbits |= 1u << ch;
                    col[ch] = 0.f;
                }
            }
            // conic pre-scaled so that power = -1/2 d^T Q d = A' dx^2 + C' dy^2 + B' dx dy
            // (A' = -A/2, B' = -B, C' = -C/2), stored times log2(e): compositing takes
            // G = 2^(stored form) without a scaling per pixel
            // .w slots: half-extents of the footprint's bounding box (compositing culls
            // whole warps with them)
            const float ci = kLog2E * id;
            st.xyo[o] = make_float4(mx, my, opac, ex);
            st.mlo[o] = make_float2(mx_lo, my_lo);
            st.con[o] = make_float4(-0.5f * (P.c * ci), P.b * ci, -0.5f * (P.a * ci), ey);
            st.col[o] = make_float4(col[0], col[1], col[2], __uint_as_float(clampbits));
        }
        st.rect[o] = rect;
        st.key[o] = ok ? __float_as_uint(P.tz) : 0xffffffffu;
    }
    return pairs;
}

// Dynamic shared memory of the projection: an mbarrier, then the block's SH rows.
constexpr int kProjThreads = 256;
constexpr size_t proj_smem_bytes(int K) { return 128 + size_t(kProjThreads) * 12 * K; }

template <int K>
__global__ void __launch_bounds__(kProjThreads, 4) project_kernel(const __grid_constant__ Views vs, Params p,
                                                                  State st)
{
    extern __shared__ __align__(128) unsigned char proj_smem[];
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(proj_smem);
    float *s_sh = reinterpret_cast<float *>(proj_smem + 128);
    // the block's SH rows are contiguous: one bulk copy streams them into shared
    // memory while the geometry is computed (rows past the live count are still
    // inside the capacity)
    const long long i0 = (long long)blockIdx.x * kProjThreads;
    const long long rows = min((long long)kProjThreads, p.cap - i0);
    const unsigned bytes = unsigned(rows) * 12u * unsigned(K);
    const bool bulk = p.sh_bulk && i0 < *p.count && (bytes & 15u) == 0;
    if (bulk) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_arrive_expect_tx(bar, bytes);
            bulk_copy_g2s(s_sh, p.sh + i0 * 3 * K, bytes, bar);
        }
        __syncthreads();
    }
    const long long i = i0 + threadIdx.x;
    unsigned long long pairs =
        i < p.cap ? project_one<K>(vs, p, st, i, bulk ? s_sh + threadIdx.x * 3 * K : nullptr, bar) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if ((threadIdx.x & 31) == 0 && pairs) atomicAdd(reinterpret_cast<unsigned long long *>(st.pairs_total), pairs);
    // the copy has landed before the block's shared memory is released
    if (bulk && threadIdx.x == 0 && !mbar_wait(bar, 0, kDefaultSpinLimit)) set_status(p.status, GSP_ERR_TIMEOUT);
}

template <int K>
void launch_project(const Views &vs, const Params &p, const State &S, long long cap, cudaStream_t s)
{
    static bool attr = false;  // once per instantiation (the size is a constant of K)
    if (!attr) {
        cudaFuncSetAttribute(project_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(proj_smem_bytes(K)));
        attr = true;
    }
    project_kernel<K><<<div_up(cap, kProjThreads), kProjThreads, proj_smem_bytes(K), s>>>(vs, p, S);
}

// Depth-sort tiles: 8 warps x 256 keys, each warp owning a contiguous slice.
constexpr int kRsThreads = 256, kRsWarps = kRsThreads / 32, kRsItems = 8;
constexpr int kRsWarpTile = 32 * kRsItems, kRsTile = kRsThreads * kRsItems;

struct SortCount {
    const int32_t *n32;  // the element count, read on the device
    __device__ long long get() const { return (long long)*n32; }
};

// -------------------------------------------------------------- depth sort
//
// Stable LSD radix sort of the depth keys of every view (blockIdx.y = view),
// four passes of 8 bits.  ds_count counts the digits of all four passes at once
// (the counts do not depend on the order of the keys).  Each pass is then one
// kernel: a block takes a ticket (tiles of kRsTile keys go in ticket order),
// ranks its tile per digit (warp-private stable ranks), publishes its digit
// counts, and walks back over the lower tickets for each digit's exclusive
// prefix (decoupled look-back).  A block publishes its count before it starts
// its own walk, and a lower ticket belongs to a block that is already running,
// so every walk ends; each poll loop is bounded all the same, and on expiry the
// pass records GSP_ERR_TIMEOUT and sets the overflow flag so that the later
// stages skip their work.
//
// Look-back word of (view, pass, tile, digit): bit 31 = inclusive prefix,
// bit 30 = the tile's own count, bits 0..29 the value (capacity < 2^30).

constexpr unsigned kLbInc = 1u << 31, kLbAgg = 1u << 30, kLbVal = kLbAgg - 1u;
constexpr long long kSortSpinLimit = 1ll << 22;

__global__ void __launch_bounds__(kRsThreads) ds_count(const uint32_t *keys, SortCount cnt, unsigned *ghist,
                                                       unsigned *state, int nb_max, long long seg)
{
    __shared__ unsigned h[4][256];
    keys += (size_t)blockIdx.y * seg;
    ghist += (size_t)blockIdx.y * 4 * 256;
    state += (size_t)blockIdx.y * 4 * nb_max * 256;  // the first pass's words of this view
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < 4 * 256; i += kRsThreads) (&h[0][0])[i] = 0;
    for (long long i = (long long)blockIdx.x * kRsThreads + tid; i < (long long)nb_max * 256;
         i += (long long)gridDim.x * kRsThreads)
        state[i] = 0;
    __syncthreads();
    const long long n = cnt.get();
    const unsigned lt = (1u << lane) - 1u;
    constexpr int kPer = 4;  // keys per thread per round, loaded before any is counted
    for (long long e0 = (long long)blockIdx.x * kRsThreads * kPer; e0 < n;
         e0 += (long long)gridDim.x * kRsThreads * kPer) {
        unsigned kv[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long e = e0 + j * kRsThreads + tid;
            kv[j] = e < n ? keys[e] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const bool ok = e0 + j * kRsThreads + tid < n;
            const unsigned k = kv[j];
            // the two low digits are spread: plain shared atomics; the two high ones
            // (exponent and leading mantissa bits of a float depth) take few values:
            // one atomic per group of equal digits in the warp
            if (ok) {
                atomicAdd(&h[0][k & 255u], 1u);
                atomicAdd(&h[1][(k >> 8) & 255u], 1u);
            }
#pragma unroll
            for (int d = 2; d < 4; ++d) {
                const unsigned dig = ok ? (k >> (8 * d)) & 255u : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, dig);
                if (ok && (peers & lt) == 0) atomicAdd(&h[d][dig], __popc(peers));
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < 4 * 256; i += kRsThreads) {
        const unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(ghist + i, c);
    }
}

__global__ void __launch_bounds__(kRsThreads) ds_pass(const uint32_t *kin, const int32_t *vin, uint32_t *kout,
                                                      int32_t *vout, SortCount cnt, int pass, const unsigned *ghist,
                                                      unsigned *state, unsigned *ticket, int nb_max, long long seg,
                                                      int32_t *overflow, int32_t *status, long long spin_limit,
                                                      int withhold)
{
    const int view = blockIdx.y;
    kin += (size_t)view * seg;
    vin += (size_t)view * seg;
    kout += (size_t)view * seg;
    vout += (size_t)view * seg;
    ghist += ((size_t)view * 4 + pass) * 256;
    unsigned *lb = state + ((size_t)view * 4 + pass) * nb_max * 256;
    __shared__ unsigned s_ticket;
    __shared__ int s_fail;
    __shared__ unsigned gbase[256], lstart[256];
    __shared__ unsigned wh[kRsWarps][256];
    __shared__ unsigned wsum[kRsWarps];
    __shared__ uint32_t sk[kRsTile];
    __shared__ int32_t sv[kRsTile];
    if (*(volatile int32_t *)overflow) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        s_ticket = atomicAdd(ticket + view * 4 + pass, 1u);
        s_fail = 0;
    }
    __syncthreads();
    const int t = int(s_ticket);
    const long long n = cnt.get();
    const long long b0 = (long long)t * kRsTile;
    if (b0 >= n) return;
    const int shift = 8 * pass;
    const long long wb = b0 + (long long)wid * kRsWarpTile;

    uint32_t key[kRsItems];
    int32_t val[kRsItems];
    unsigned dig[kRsItems], rank[kRsItems];
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        const long long e = wb + j * 32 + lane;
        const bool ok = e < n;
        key[j] = ok ? kin[e] : 0u;
        val[j] = ok ? vin[e] : 0;
        dig[j] = ok ? ((key[j] >> shift) & 255u) : 256u;
    }
    for (int k = lane; k < 256; k += 32) wh[wid][k] = 0;
    __syncwarp();
    // warp-private stable ranks, items in (j, lane) order
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        const unsigned d = dig[j];
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        unsigned before = 0;
        if (lane == leader && d < 256u) {
            before = wh[wid][d];
            wh[wid][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rank[j] = before + __popc(peers & ((1u << lane) - 1u));
        __syncwarp();
    }
    __syncthreads();
    // digit tid: the warps' offsets and the tile's count, published at once
    unsigned tot = 0;
    for (int w = 0; w < kRsWarps; ++w) {
        const unsigned c = wh[w][tid];
        wh[w][tid] = tot;
        tot += c;
    }
    volatile unsigned *vlb = lb;
    // (test hook: tile 0 withholds its word, so every later tile's walk runs out)
    if (!(withhold && t == 0)) vlb[(size_t)t * 256 + tid] = (t == 0 ? kLbInc : kLbAgg) | tot;
    // tile-local digit starts; digit starts over the view
    unsigned gstart;
    {
        unsigned inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        unsigned base = 0;
        for (int w = 0; w < wid; ++w) base += wsum[w];
        lstart[tid] = base + inc - tot;
        const unsigned x = ghist[tid];
        inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        __syncthreads();
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        base = 0;
        for (int w = 0; w < wid; ++w) base += wsum[w];
        gstart = base + inc - x;
    }
    // look-back: the keys with digit tid in the lower tiles
    // (four lower tiles per round trip: tile 0 always holds an inclusive word)
    unsigned prefix = 0;
    if (t > 0) {
        int j = t - 1;
        long long polls = 0;
        bool done = false;
        while (!done) {
            unsigned w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = j - q >= 0 ? unsigned(vlb[(size_t)(j - q) * 256 + tid]) : unsigned(kLbInc);
            int used = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (done || used < q) break;  // stopped earlier in this round
                if (!(w[q] & (kLbInc | kLbAgg))) break;  // not published yet: poll again from here
                prefix += w[q] & kLbVal;
                used = q + 1;
                if (w[q] & kLbInc) done = true;
            }
            j -= used;
            if (!done && used == 0 && ++polls > spin_limit) {
                s_fail = 1;
                break;
            }
        }
        vlb[(size_t)t * 256 + tid] = kLbInc | (prefix + tot);
    }
    if (pass < 3) lb[(size_t)nb_max * 256 + (size_t)t * 256 + tid] = 0;  // the next pass's word
    gbase[tid] = gstart + prefix;
    __syncthreads();
    if (s_fail) {
        if (tid == 0) {
            set_status(status, GSP_ERR_TIMEOUT);
            atomicExch(overflow, 1);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        if (dig[j] < 256u) {
            const unsigned p = lstart[dig[j]] + wh[wid][dig[j]] + rank[j];
            sk[p] = key[j];
            sv[p] = val[j];
        }
    }
    __syncthreads();
    const int cnt_blk = int(min((long long)kRsTile, n - b0));
    for (int i = tid; i < cnt_blk; i += kRsThreads) {
        const uint32_t k = sk[i];
        const unsigned d = (k >> shift) & 255u;
        const long long pos = (long long)gbase[d] + (i - lstart[d]);
        if (!GSP_BOUND(pos, n, status)) continue;
        kout[pos] = k;
        vout[pos] = sv[i];
    }
}

// ---------------------------------------------------------------- binning
//
// Stable two-level counting sort of the depth-ordered Gaussians into per-tile
// lists (no sort over the pairs).  Tiles are grouped into 8x8 supertiles.
//   level 1  the depth order of each view is partitioned, stably, into one
//            list per supertile the Gaussian's tile rectangle touches
//   level 2  each supertile list is partitioned, stably, into its 64 tile
//            lists, which come out contiguous (tile-major) in `ids`
// Work is cut into warp chunks of 128 ranks (level 1) or 256 entries of one
// supertile list (level 2).  Each level counts per (chunk, bin), scans the
// counts per bin over the chunks, and scatters with the chunk's cursors:
//   l1_count    per chunk: supertile counts (shared-memory atomics, order-free)
//   l1_scan     one block per supertile: chunk offsets inside its list
//   bin_tops    one block: list starts, level-2 chunk bases, capacity check
//   l1_scatter  per chunk: warp-ordered scatter of the ids (a min-reduction
//               walks the supertiles of the warp's 32 Gaussians in ascending
//               order; lanes sharing a supertile write in lane = rank order)
//   l2_count    per chunk: the 64-bit tile mask of each entry (rows of the
//               rectangle inside the supertile, culled by the exact column
//               intervals), stored; per-tile counts from the transposed masks
//   l2_scan     one block per supertile: chunk offsets per tile, list lengths
//   tile_scan   one block: list starts of all tiles
//   l2_scatter  per chunk: for each tile and round, a ballot gives every lane
//               its slot; each store writes a contiguous run of the list.
//               Only the first st.prefix positions of each list are written
//               (a chunk that lies wholly past them is skipped): the forward
//               compositing stops once every pixel of a tile has saturated,
//               which on dense tiles happens within a few hundred entries.
//               Tiles that need more are marked by the compositing; a second
//               pass (rest = 1) then writes the remainder of their lists.

constexpr int kSuper = 8;                 // supertile edge, in tiles
constexpr int kL1Ranks = 128;             // ranks per level-1 warp chunk
constexpr int kL1Rounds = kL1Ranks / 32;
constexpr int kBinRanks = 256;            // supertile entries per level-2 warp chunk
constexpr int kBinRounds = kBinRanks / 32;
constexpr int kBinWarps = 4, kBinThreads = kBinWarps * 32;
constexpr int kMaxSuper = 2048;           // supertiles per view (shared-memory tables)

__device__ __forceinline__ void rect_unpack(uint2 r, int &tx0, int &ty0, int &tx1, int &ty1)
{
    tx0 = int(r.x & 0xffffu); ty0 = int(r.x >> 16); tx1 = int(r.y & 0xffffu); ty1 = int(r.y >> 16);
}

__device__ __forceinline__ int find_view_super(const Views &vs, int gs)
{
    int v = 0;
    while (v + 1 < vs.n && vs.v[v + 1].super_base <= gs) ++v;
    return v;
}

// Columns [lo, hi] of tile row ty0 + yy that the 1/255 ellipse reaches (lo > hi: none).
__device__ __forceinline__ void row_interval(const uchar2 *ri, int yy, int tx0, int tx1, int &lo, int &hi)
{
    lo = tx0;
    hi = tx1;
    if (yy < kRowCap) {
        const uchar2 iv = ri[yy];
        lo = tx0 + int(iv.x);
        hi = iv.y == 255 ? tx1 : tx0 + int(iv.y);
    }
}

// Tiles of supertile (sx, sy) the ellipse reaches: bit (ty - 8 sy) * 8 + (tx - 8 sx).
__device__ __forceinline__ unsigned long long entry_mask(uint2 rc, const uchar2 *ri, int sx, int sy)
{
    int tx0, ty0, tx1, ty1;
    rect_unpack(rc, tx0, ty0, tx1, ty1);
    const int bx = sx * kSuper, by = sy * kSuper;
    unsigned long long m = 0;
#pragma unroll
    for (int r = 0; r < kSuper; ++r) {
        const int ty = by + r;
        if (ty < ty0 || ty > ty1) continue;
        int lo, hi;
        row_interval(ri, ty - ty0, tx0, tx1, lo, hi);
        lo = max(lo, bx);
        hi = min(hi, bx + kSuper - 1);
        if (lo <= hi)
            m |= (unsigned long long)((0xffu >> (kSuper - 1 - (hi - lo))) << (lo - bx)) << (r * kSuper);
    }
    return m;
}

// Level-1 chunk `task` (over all views): its view, first rank and rank count.
struct L1Task {
    int v, chunk, r0, cnt;
};

__device__ __forceinline__ L1Task l1_task(int task, int n)
{
    const int nch = (n + kL1Ranks - 1) / kL1Ranks;
    L1Task t;
    t.v = task / nch;
    t.chunk = task - t.v * nch;
    t.r0 = t.chunk * kL1Ranks;
    t.cnt = min(kL1Ranks, n - t.r0);
    return t;
}

__global__ void __launch_bounds__(kBinThreads) l1_count(const __grid_constant__ Views vs, State st, long long cap)
{
    extern __shared__ unsigned l1_tab[];  // [kBinWarps][smax]
    if (*st.overflow) return;
    const int n = *st.n_dev;
    const int nch = (n + kL1Ranks - 1) / kL1Ranks;
    const int ntask = nch * vs.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned *tab = l1_tab + wid * vs.smax;
    for (int s = lane; s < vs.smax; s += 32) tab[s] = 0;
    __syncwarp();
    for (int task = blockIdx.x * kBinWarps + wid; task < ntask; task += gridDim.x * kBinWarps) {
        const L1Task t = l1_task(task, n);
        const ViewP &V = vs.v[t.v];
        const int32_t *sorted = st.val + (size_t)t.v * cap;
        const uint2 *rect = st.rect + (size_t)t.v * cap;
        for (int k = 0; k < kL1Rounds; ++k) {
            const int r = 32 * k + lane;
            if (r >= t.cnt) break;
            const uint2 rc = rect[sorted[t.r0 + r]];
            int tx0, ty0, tx1, ty1;
            rect_unpack(rc, tx0, ty0, tx1, ty1);
            if (tx1 < tx0) continue;
            for (int sy = ty0 / kSuper; sy <= ty1 / kSuper; ++sy)
                for (int sx = tx0 / kSuper; sx <= tx1 / kSuper; ++sx)
                    if (GSP_BOUND(sy * V.sx + sx, vs.smax, st.status)) atomicAdd(&tab[sy * V.sx + sx], 1u);
        }
        __syncwarp();
        const int S = V.sx * V.sy;
        for (int s = lane; s < S; s += 32) {
            st.count1[(size_t)(V.super_base + s) * st.nch1_max + t.chunk] = tab[s];
            tab[s] = 0;
        }
        __syncwarp();
    }
}

// Block-wide exclusive scan of one value per thread (NT threads); returns the
// exclusive prefix and stores the total in *total.  wsum: NT / 32 words.
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long x, unsigned long long *wsum,
                                                              unsigned long long *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned long long base = 0, all = 0;
    for (int w = 0; w < NT / 32; ++w) {
        if (w < wid) base += wsum[w];
        all += wsum[w];
    }
    *total = all;
    __syncthreads();
    return base + inc - x;
}

// One block per supertile (all views): offsets of the chunks inside its list.
constexpr int kScanThreads = 1024;  // l1_scan / l2_scan: one block per supertile

// Whether this block is the last of the grid to arrive (its writes, and all
// earlier blocks', are then visible to it).
__device__ __forceinline__ bool last_block(unsigned *ticket)
{
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

__device__ void bin_tops(int total_super, State st, int32_t *status);
__device__ void tile_scan(int total_tiles, State st, int32_t *status);

__global__ void __launch_bounds__(kScanThreads) l1_scan(const __grid_constant__ Views vs, State st, int32_t *status)
{
    __shared__ unsigned long long wsum[kScanThreads / 32];
    if (!*st.overflow) {
        const int gs = blockIdx.x;
        const int n = *st.n_dev;
        const int nch = (n + kL1Ranks - 1) / kL1Ranks;
        unsigned *row = st.count1 + (size_t)gs * st.nch1_max;
        const int q = (nch + kScanThreads - 1) / kScanThreads;
        const int c0 = threadIdx.x * q, c1 = min(c0 + q, nch);
        // (8 loads in flight per step: a running sum over dependent loads
        // would wait for each one)
        unsigned long long sum = 0;
        for (int c = c0; c < c1; c += 8) {
            unsigned x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = c + u < c1 ? row[c + u] : 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += x[u];
        }
        unsigned long long total;
        unsigned long long run = block_excl_scan<kScanThreads>(sum, wsum, &total);
        for (int c = c0; c < c1; c += 8) {
            unsigned x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = c + u < c1 ? row[c + u] : 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (c + u < c1) row[c + u] = unsigned(run);
                run += x[u];
            }
        }
        if (threadIdx.x == 0) st.len1[gs] = unsigned(total);
    }
    // the last block: starts of the supertile lists, level-2 chunk bases
    if (last_block(st.scan_ticket)) bin_tops(vs.total_super, st, status);
}

// Starts of the supertile lists, level-2 chunk bases, capacity check (one
// block of kScanThreads, the last of l1_scan).
__device__ void bin_tops(int total_super, State st, int32_t *status)
{
    __shared__ unsigned long long wsum[2][32];
    __shared__ unsigned long long carry[2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    const bool over0 = *st.overflow;
    for (int b0 = 0; b0 < total_super; b0 += 1024) {
        const int gs = b0 + threadIdx.x;
        const unsigned long long len = (!over0 && gs < total_super) ? __ldcg(st.len1 + gs) : 0;
        const unsigned long long nc = (len + kBinRanks - 1) / kBinRanks;
        unsigned long long a = len, b = nc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long ya = __shfl_up_sync(0xffffffffu, a, o);
            const unsigned long long yb = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += ya; b += yb; }
        }
        if (lane == 31) { wsum[0][wid] = a; wsum[1][wid] = b; }
        __syncthreads();
        unsigned long long ba = 0, bb = 0, ta = 0, tb = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < wid) { ba += wsum[0][w]; bb += wsum[1][w]; }
            ta += wsum[0][w];
            tb += wsum[1][w];
        }
        const unsigned long long ca = carry[0], cb = carry[1];
        __syncthreads();
        if (gs < total_super) {
            st.list1_start[gs] = unsigned(ca + ba + a - len);
            st.chunk2_base[gs] = unsigned(cb + bb + b - nc);
        }
        if (threadIdx.x == 0) { carry[0] = ca + ta; carry[1] = cb + tb; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st.chunk2_base[total_super] = over0 ? 0u : unsigned(carry[1]);
        const int over = over0 || *st.pairs_total > st.pair_cap || (long long)carry[0] > st.pair_cap;
        *st.overflow = over;
        if (over) {
            st.chunk2_base[total_super] = 0;
            set_status(status, GSP_ERR_CAPACITY);
        }
    }
}

__global__ void __launch_bounds__(kBinThreads) l1_scatter(const __grid_constant__ Views vs, State st, long long cap)
{
    extern __shared__ unsigned l1_cur[];  // [kBinWarps][smax]
    if (*st.overflow) return;
    const int n = *st.n_dev;
    const int nch = (n + kL1Ranks - 1) / kL1Ranks;
    const int ntask = nch * vs.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned *cur = l1_cur + wid * vs.smax;
    for (int task = blockIdx.x * kBinWarps + wid; task < ntask; task += gridDim.x * kBinWarps) {
        const L1Task t = l1_task(task, n);
        const ViewP &V = vs.v[t.v];
        const int S = V.sx * V.sy;
        for (int s = lane; s < S; s += 32)
            cur[s] = st.list1_start[V.super_base + s] +
                     st.count1[(size_t)(V.super_base + s) * st.nch1_max + t.chunk];
        __syncwarp();
        const int32_t *sorted = st.val + (size_t)t.v * cap;
        const uint2 *rect = st.rect + (size_t)t.v * cap;
        for (int k = 0; k < kL1Rounds; ++k) {
            if (32 * k >= t.cnt) break;
            const int r = 32 * k + lane;
            int g = -1;
            int sx0 = 0, sx1 = -1, sy1 = -1, csx = 0, csy = 0;
            bool live = false;
            if (r < t.cnt) {
                g = sorted[t.r0 + r];
                int tx0, ty0, tx1, ty1;
                rect_unpack(rect[g], tx0, ty0, tx1, ty1);
                if (tx1 >= tx0) {
                    sx0 = tx0 / kSuper; sx1 = tx1 / kSuper; sy1 = ty1 / kSuper;
                    csx = sx0; csy = ty0 / kSuper;
                    live = true;
                }
            }
            // supertiles of the round in ascending order; every lane's current
            // cell is its smallest unwritten one, so the minimum is shared by all
            // lanes whose rectangle contains it
            for (;;) {
                const unsigned key = live ? unsigned(csy * V.sx + csx) : 0xffffffffu;
                const unsigned smin = __reduce_min_sync(0xffffffffu, key);
                if (smin == 0xffffffffu) break;
                const bool mine = key == smin;
                const unsigned bal = __ballot_sync(0xffffffffu, mine);
                unsigned base = 0;
                if (lane == 0 && GSP_BOUND(smin, vs.smax, st.status)) {
                    base = cur[smin];
                    cur[smin] = base + __popc(bal);
                }
                base = __shfl_sync(0xffffffffu, base, 0);
                if (mine) {
                    if (GSP_BOUND(base + __popc(bal & lt), st.pair_cap, st.status)) st.id1[base + __popc(bal & lt)] = g;
                    if (++csx > sx1) {
                        csx = sx0;
                        if (++csy > sy1) live = false;
                    }
                }
            }
        }
        __syncwarp();
    }
}

// 32 x 32 bit-matrix transpose across the warp: lane L returns the word whose
// bit i is bit L of lane i's x.  Stage j exchanges, between lanes L and L ^ j,
// the off-diagonal j x j blocks of every 2j x 2j block: a rotate by j (left in
// the lower lane, right in the upper one) moves the partner's block into place
// and a mask merge keeps the lane's own diagonal block.
__device__ __forceinline__ unsigned warp_transpose32(unsigned x, int lane)
{
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const unsigned m = j == 16 ? 0x0000ffffu : j == 8 ? 0x00ff00ffu : j == 4 ? 0x0f0f0f0fu
                           : j == 2 ? 0x33333333u : 0x55555555u;
        const bool upper = lane & j;
        const unsigned y = __shfl_xor_sync(0xffffffffu, x, j);
        const unsigned t = __funnelshift_l(y, y, upper ? 32 - j : j);
        const unsigned keep = upper ? ~m : m;
        x = (x & keep) | (t & ~keep);
    }
    return x;
}

// Level-2 chunk c: its supertile (largest gs with chunk2_base[gs] <= c).
__device__ __forceinline__ int l2_super(const State &st, int total_super, unsigned c)
{
    int lo = 0, hi = total_super;  // chunk2_base[lo] <= c < chunk2_base[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (st.chunk2_base[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kBinThreads) l2_count(const __grid_constant__ Views vs, State st, long long cap)
{
    if (*st.overflow) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned nchunk = st.chunk2_base[vs.total_super];
    for (unsigned c = blockIdx.x * kBinWarps + wid; c < nchunk; c += gridDim.x * kBinWarps) {
        const int gs = l2_super(st, vs.total_super, c);
        if (lane == 0) st.chunk_super[c] = gs;  // for l2_scatter
        const int v = find_view_super(vs, gs);
        const ViewP &V = vs.v[v];
        const int s = gs - V.super_base;
        const int sy = s / V.sx, sx = s - sy * V.sx;
        const unsigned e0 = st.list1_start[gs] + (c - st.chunk2_base[gs]) * kBinRanks;
        const unsigned e1 = st.list1_start[gs] + st.len1[gs];
        const uint2 *rect = st.rect + (size_t)v * cap;
        const uchar2 *rowint = st.rowint + (size_t)v * cap * kRowCap;
        unsigned long long m[kBinRounds];
#pragma unroll
        for (int k = 0; k < kBinRounds; ++k) {
            const unsigned e = e0 + 32 * k + lane;
            m[k] = 0;
            if (e < e1 && GSP_BOUND(e, st.pair_cap, st.status)) {
                const int g = st.id1[e];
                if (GSP_BOUND(g, cap, st.status)) {
                    m[k] = entry_mask(rect[g], rowint + (size_t)g * kRowCap, sx, sy);
                    st.mask1[e] = m[k];
                }
            }
        }
        // per-tile counts: after the transpose lane L holds, per round, the
        // entries of tile L (low half) and of tile L + 32 (high half)
        unsigned mc0 = 0, mc1 = 0;
#pragma unroll
        for (int k = 0; k < kBinRounds; ++k) {
            mc0 += __popc(warp_transpose32(unsigned(m[k]), lane));
            mc1 += __popc(warp_transpose32(unsigned(m[k] >> 32), lane));
        }
        st.count2[(size_t)c * 64 + lane] = mc0;
        st.count2[(size_t)c * 64 + 32 + lane] = mc1;
    }
}

// Global tile of bit b of supertile (sx, sy) of view V, or -1 outside the view.
__device__ __forceinline__ int super_tile(const ViewP &V, int sx, int sy, int b)
{
    const int tx = sx * kSuper + (b & (kSuper - 1)), ty = sy * kSuper + b / kSuper;
    return (tx < V.tiles_x && ty < V.tiles_y) ? V.tile_base + ty * V.tiles_x + tx : -1;
}

// One block per supertile: offsets of its chunks inside each tile's list, and
// the tiles' list lengths.  Thread (group, b): tile b over a quarter of the chunks.
__global__ void __launch_bounds__(kScanThreads) l2_scan(const __grid_constant__ Views vs, State st, int32_t *status)
{
    constexpr int kGroups = kScanThreads / 64;
    __shared__ unsigned part[kGroups][64];
    const int gs = blockIdx.x;
    const int v = find_view_super(vs, gs);
    const ViewP &V = vs.v[v];
    const int s = gs - V.super_base;
    const int sy = s / V.sx, sx = s - sy * V.sx;
    const int b = threadIdx.x & 63, grp = threadIdx.x >> 6;
    const bool over = *st.overflow;
    const unsigned cb0 = over ? 0u : st.chunk2_base[gs], cb1 = over ? 0u : st.chunk2_base[gs + 1];
    const unsigned nch = cb1 - cb0, q = (nch + kGroups - 1) / kGroups;
    const unsigned c0 = cb0 + grp * q, c1 = min(c0 + q, cb1);
    // (8 loads in flight per step, as in l1_scan)
    unsigned sum = 0;
    for (unsigned c = c0; c < c1; c += 8) {
        unsigned x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = c + u < c1 ? st.count2[(size_t)(c + u) * 64 + b] : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) sum += x[u];
    }
    part[grp][b] = sum;
    __syncthreads();
    unsigned run = 0;
    for (int g2 = 0; g2 < grp; ++g2) run += part[g2][b];
    for (unsigned c = c0; c < c1; c += 8) {
        unsigned x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = c + u < c1 ? st.count2[(size_t)(c + u) * 64 + b] : 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (c + u < c1) st.count2[(size_t)(c + u) * 64 + b] = run;
            run += x[u];
        }
    }
    if (grp == kGroups - 1) {
        const int gt = super_tile(V, sx, sy, b);
        if (gt >= 0) st.tile_len[gt] = run;
    }
    // the last block: starts of the tile lists and the forward's tile order
    if (last_block(st.scan_ticket + 1)) tile_scan(vs.total_tiles, st, status);
}

// 8-bit logarithmic bucket of a work estimate: 3 bits of mantissa under the
// position of the leading one.
__device__ __forceinline__ unsigned work_bucket(unsigned v)
{
    if (v == 0) return 0;
    const int l = 31 - __clz(v);
    const unsigned f = l >= 3 ? (v >> (l - 3)) & 7u : (v << (3 - l)) & 7u;
    return unsigned(l) * 8u + f;
}

// One block of 1024 threads: tiles in descending order of work (counting sort
// on work_bucket), so that the longest tiles are dispatched first and the
// launch does not end on a tail of heavy tiles.
__device__ void order_tiles_desc(const unsigned *work, int total_tiles, int32_t *order)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid < 256) hist[tid] = 0;
    __syncthreads();
    for (int t = tid; t < total_tiles; t += blockDim.x) atomicAdd(&hist[255u - work_bucket(__ldcg(work + t))], 1u);
    __syncthreads();
    unsigned x = 0, inc = 0;
    if (tid < 256) {
        x = hist[tid];
        inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[wid] = inc;
    }
    __syncthreads();
    if (tid < 256) {
        unsigned base = 0;
        for (int w = 0; w < wid; ++w) base += wsum[w];
        hist[tid] = base + inc - x;
    }
    __syncthreads();
    for (int t = tid; t < total_tiles; t += blockDim.x)
        order[atomicAdd(&hist[255u - work_bucket(__ldcg(work + t))], 1u)] = t;
}

// Exclusive scan of the tile list lengths into list starts (one block of
// kScanThreads, the last of l2_scan); the total is checked against the pair
// capacity once more before any id is written.  Each tile's list is then
// written up to its first st.prefix entries (tile_avail).
__device__ void tile_scan(int total_tiles, State st, int32_t *status)
{
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < total_tiles; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const unsigned long long x = i < total_tiles ? __ldcg(st.tile_len + i) : 0;
        unsigned long long inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        unsigned long long wb = 0, all = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < wid) wb += wsum[w];
            all += wsum[w];
        }
        const unsigned long long c0 = carry;
        __syncthreads();
        if (i < total_tiles) {
            st.tile_start[i] = unsigned(c0 + wb + inc - x);
            st.tile_avail[i] = unsigned(min(x, (unsigned long long)st.prefix));
        }
        if (threadIdx.x == 0) carry = c0 + all;
        __syncthreads();
    }
    if (threadIdx.x == 0 && (long long)carry > st.pair_cap) {
        *st.overflow = 1;
        set_status(status, GSP_ERR_CAPACITY);
    }
    order_tiles_desc(st.tile_len, total_tiles, st.order_fwd);
}

// One block: the adjoint's tile order, by the forward's last-contributor positions.
__global__ void __launch_bounds__(1024) tile_order_bwd(int total_tiles, State st)
{
    order_tiles_desc(st.tile_work, total_tiles, st.order_bwd);
}

// rest = 0: every tile's entries at list positions below its prefix
// (tile_avail); rest = 1 (after the forward compositing): the remaining
// entries of the tiles the forward marked for a redo, nothing when it marked
// none.  A work item is one chunk and one group of kScatterTiles of its
// supertile's tiles (lane t: tile t of the group), so that the few chunks with
// positions to write (the first of each supertile list) spread over many
// warps; an item whose tiles need nothing from its chunk is skipped before
// the chunk's entries are read.
constexpr int kScatterTiles = 16;
constexpr int kScatterGroups = 64 / kScatterTiles;

__global__ void __launch_bounds__(kBinThreads) l2_scatter(const __grid_constant__ Views vs, State st, int rest)
{
    if (*st.overflow) return;
    if (rest && __ldcg(st.redo_count) == 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned nitem = st.chunk2_base[vs.total_super] * kScatterGroups;
    for (unsigned it = blockIdx.x * kBinWarps + wid; it < nitem; it += gridDim.x * kBinWarps) {
        const unsigned c = it / kScatterGroups;
        const int grp = int(it % kScatterGroups);
        const int gs = st.chunk_super[c];
        if (!GSP_BOUND(gs, vs.total_super, st.status)) continue;
        if (rest && __ldcg(st.super_redo + gs) == 0) continue;
        const int v = find_view_super(vs, gs);
        const ViewP &V = vs.v[v];
        const int s = gs - V.super_base;
        const int sy = s / V.sx, sx = s - sy * V.sx;
        // lane t < kScatterTiles: tile t of the group, the chunk's first list
        // position in it and the window [lo, hi) of positions this pass writes
        const int gt = lane < kScatterTiles ? super_tile(V, sx, sy, grp * kScatterTiles + lane) : -1;
        unsigned cur = 0, lo = 0, hi = 0;
        if (gt >= 0) {
            const unsigned ts = st.tile_start[gt];
            cur = ts + st.count2[(size_t)c * 64 + grp * kScatterTiles + lane];
            if (!rest) {
                lo = ts;
                hi = ts + st.tile_avail[gt];
            } else if (__ldcg(st.tile_redo + gt)) {
                lo = ts + st.tile_avail[gt];
                hi = ts + st.tile_len[gt];
            }
        }
        const unsigned want = __ballot_sync(0xffffffffu, cur < hi);
        if (want == 0) continue;
        const unsigned e0 = st.list1_start[gs] + (c - st.chunk2_base[gs]) * kBinRanks;
        const unsigned e1 = st.list1_start[gs] + st.len1[gs];
        int g[kBinRounds];
        unsigned mh[kBinRounds];
        unsigned any = 0;
#pragma unroll
        for (int k = 0; k < kBinRounds; ++k) {
            const unsigned e = e0 + 32 * k + lane;
            g[k] = 0;
            mh[k] = 0;
            if (e < e1 && GSP_BOUND(e, st.pair_cap, st.status)) {
                g[k] = st.id1[e];
                mh[k] = unsigned(st.mask1[e] >> (grp * kScatterTiles)) & ((1u << kScatterTiles) - 1u);
            }
            any |= mh[k];
        }
        unsigned present = __reduce_or_sync(0xffffffffu, any) & want;
        while (present) {
            const int b = __ffs(present) - 1;
            present &= present - 1;
            unsigned base = __shfl_sync(0xffffffffu, cur, b);
            const unsigned wlo = __shfl_sync(0xffffffffu, lo, b), whi = __shfl_sync(0xffffffffu, hi, b);
#pragma unroll
            for (int k = 0; k < kBinRounds; ++k) {
                const bool bit = (mh[k] >> b) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                const unsigned pos = base + __popc(bal & lt);
                if (bit && pos >= wlo && pos < whi && GSP_BOUND(pos, st.pair_cap, st.status)) st.ids[pos] = g[k];
                base += __popc(bal);
                if (base >= whi) break;  // warp-uniform: the window is full
            }
        }
    }
}

// ------------------------------------------------------------- compositing

// Pixel layout of a compositing block (one 16x16 tile, kTilePix / PPT threads):
// each warp covers an 8-column x 4 PPT-row block (lanes 8 wide, 4 tall, each a
// vertical run of PPT pixels), the warps 2 across.  A compact warp footprint
// keeps the warp's pixels close, so fewer Gaussians reach only some of them.
template <int PPT>
struct WarpBlock {
    int x, y0;            // the thread's column and first row (image pixels)
    float wcx, wcy;       // centre of the warp's pixel centres
    static constexpr float whw = 3.5f, whh = 2.f * PPT - 0.5f;  // their half-extents
    __device__ __forceinline__ WarpBlock(int txx, int tyy, int tid)
    {
        const int lane = tid & 31, wid = tid >> 5;
        const int wx = wid & 1, wy = wid >> 1;
        x = txx * kTile + wx * 8 + (lane & 7);
        y0 = tyy * kTile + (wy * 4 + (lane >> 3)) * PPT;
        wcx = txx * kTile + wx * 8 + 4.f;
        wcy = tyy * kTile + wy * 4 * PPT + 2.f * PPT;
    }
};

struct Alpha {
    float G, raw, alpha, dx, dy, dxx, dyy, dxy;
    bool pass;
};

// Identical in the forward and the backward kernel (explicitly rounded ops),
// so both take the same 1/255 decision.  The exponential is evaluated for every
// lane (a branch around it costs more than the MUFU op it saves).
__device__ __forceinline__ Alpha eval_alpha(float4 xyo, float2 lo, float4 con, float px, float py)
{
    Alpha r;
    // d = pixel centre - (hi + lo); px - hi is exact when px and hi are within a
    // factor of two (Sterbenz), else off by half an ulp of a small coordinate
    r.dx = __fsub_rn(__fsub_rn(px, xyo.x), lo.x);
    r.dy = __fsub_rn(__fsub_rn(py, xyo.y), lo.y);
    r.dxx = __fmul_rn(r.dx, r.dx);
    r.dyy = __fmul_rn(r.dy, r.dy);
    r.dxy = __fmul_rn(r.dx, r.dy);
    const float power2 = __fmaf_rn(con.x, r.dxx, __fmaf_rn(con.z, r.dyy, __fmul_rn(con.y, r.dxy)));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r.G) : "f"(power2));
    r.raw = __fmul_rn(xyo.z, r.G);
    r.alpha = fminf(kAlphaMax, r.raw);
    r.pass = r.alpha >= kAlphaMin;
    return r;
}

__device__ __forceinline__ float target_value(const ViewP &V, int x, int y, int ch)
{
    return __fdiv_rn(float(V.tgt[(long long)y * V.tgt_pitch + 3 * x + ch]), 255.f);
}

// Forward compositing: one block per 16x16 tile, each thread a vertical run
// of PPT pixels.  The tile's list is staged through shared memory in batches
// of BATCH Gaussians; the block leaves when every pixel has stopped.
// Only a prefix of each list has been written (tile_avail: the first
// st.prefix entries); a tile that reaches its end with a pixel still running
// saves every pixel's state (colour, T, last, stopped) in the outputs, is
// marked and leaves.  REDO: the blocks resume the marked tiles from their
// saved state over the rest of their lists (written meanwhile by l2_scatter
// with rest = 1), block b the tiles b, b + grid, ...  Every pixel thus sees
// the same Gaussians in the same order with the same arithmetic as over
// the whole list.

template <int PPT, int BATCH, bool CULL, bool REDO>
__global__ void __launch_bounds__(kTilePix / PPT) composite_fwd(const __grid_constant__ Views vs, State st,
                                                                long long cap, const float *edge, float *rgb_out,
                                                                float *T_out, int32_t *last_out, float *score)
{
    constexpr int NT = kTilePix / PPT;
    __shared__ float4 s_xyo[BATCH], s_con[BATCH], s_col[BATCH];
    __shared__ float2 s_mlo[BATCH];
    __shared__ int32_t s_id[BATCH];
    __shared__ float s_score[BATCH];
    __shared__ float s_red[NT / 32];
    __shared__ unsigned s_maxlast;
    __shared__ unsigned long long s_contrib;
    if (*st.overflow) return;
    // first pass: block b composites tile order_fwd[b]; redo pass: a smaller
    // grid loops over the marked tiles
    for (int item = blockIdx.x;; item += gridDim.x) {
        int gt;
        if constexpr (REDO) {
            if (item >= int(__ldcg(st.redo_count))) return;
            gt = __ldcg(st.redo_list + item);
            __syncthreads();  // the previous tile's shared state is no longer read
        } else {
            gt = st.order_fwd[item];
        }
        const int v = find_view(vs, gt);
        const ViewP &V = vs.v[v];
        const int lt = gt - V.tile_base;
        const int tyy = lt / V.tiles_x, txx = lt - tyy * V.tiles_x;
        const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
        const WarpBlock<PPT> wb(txx, tyy, tid);
        const int x = wb.x, y0 = wb.y0;
        const float wcx = wb.wcx, wcy = wb.wcy, whw = wb.whw, whh = wb.whh;
        const float px = x + 0.5f;
        const int len_full = int(st.tile_len[gt]);
        const int avail = int(st.tile_avail[gt]);
        const int len = REDO ? len_full : avail;
        const int32_t *list = st.ids + st.tile_start[gt];
        const float4 *xyo = st.xyo + (size_t)v * cap, *con = st.con + (size_t)v * cap, *col = st.col + (size_t)v * cap;
        const float2 *mlo = st.mlo + (size_t)v * cap;
        if (tid == 0) {
            s_maxlast = 0;
            s_contrib = 0;
        }
        __syncthreads();
        unsigned ncontrib = 0;

        float T[PPT], C0[PPT], C1[PPT], C2[PPT], E[PPT];
        int last[PPT];
        bool done[PPT];
#pragma unroll
        for (int m = 0; m < PPT; ++m) {
            const int y = y0 + m;
            const bool inside = x < V.w && y < V.h;
            T[m] = 1.f; C0[m] = C1[m] = C2[m] = 0.f; last[m] = 0;
            done[m] = !inside;
            E[m] = (edge && inside) ? edge[V.pix_off + (long long)y * V.w + x] : 0.f;
            if (REDO && inside) {  // the state the first pass saved at the end of the prefix
                const long long pid = V.pix_off + (long long)y * V.w + x;
                C0[m] = rgb_out[3 * pid];
                C1[m] = rgb_out[3 * pid + 1];
                C2[m] = rgb_out[3 * pid + 2];
                T[m] = T_out[pid];
                const int l = last_out[pid];
                last[m] = l & 0x7fffffff;
                done[m] = l < 0;
            }
        }
        for (int b = REDO ? avail : 0; b < len; b += BATCH) {
            bool all = true;
#pragma unroll
            for (int m = 0; m < PPT; ++m) all = all && done[m];
            if (__syncthreads_count(all) == NT) break;
            for (int q = tid; q < BATCH; q += NT) {
                const int k = b + q;
                if (k < len) {
                    int id = 0;
                    if (GSP_BOUND((long long)st.tile_start[gt] + k, st.pair_cap, st.status)) id = list[k];
                    if (!GSP_BOUND(id, cap, st.status)) id = 0;
                    s_id[q] = id;
                    s_xyo[q] = xyo[id];
                    s_mlo[q] = mlo[id];
                    s_con[q] = con[id];
                    s_col[q] = col[id];
                }
                if (score) s_score[q] = 0.f;
            }
            __syncthreads();
            const int cnt = min(BATCH, len - b);
            for (int j = 0; j < cnt; ++j) {
                const float4 gx = s_xyo[j], gc = s_con[j];
                // the footprint's bounding box misses every pixel of the warp (warp-uniform)
                if (CULL && (fabsf(gx.x - wcx) > gx.w + whw || fabsf(gx.y - wcy) > gc.w + whh)) continue;
                float sv = 0.f;
#pragma unroll
                for (int m = 0; m < PPT; ++m) {
                    if (done[m]) continue;
                    const Alpha a = eval_alpha(gx, s_mlo[j], gc, px, y0 + m + 0.5f);
                    if (!a.pass) continue;
                    const float Tn = __fmul_rn(T[m], __fsub_rn(1.f, a.alpha));
                    if (Tn < kTMin) {
                        done[m] = true;
                        continue;
                    }
                    ++ncontrib;
                    const float w = __fmul_rn(a.alpha, T[m]);
                    const float4 c = s_col[j];
                    C0[m] = __fmaf_rn(c.x, w, C0[m]);
                    C1[m] = __fmaf_rn(c.y, w, C1[m]);
                    C2[m] = __fmaf_rn(c.z, w, C2[m]);
                    T[m] = Tn;
                    last[m] = b + j + 1;
                    sv = __fmaf_rn(w, E[m], sv);
                }
                if (score && __any_sync(0xffffffffu, sv != 0.f)) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
                    if (lane == 0) atomicAdd(&s_score[j], sv);
                }
            }
            __syncthreads();
            if (score)
                for (int q = tid; q < cnt; q += NT)
                    if (s_score[q] != 0.f) atomicAdd(&score[s_id[q]], s_score[q]);
        }
        if (!REDO && len < len_full) {
            // the written prefix ran out with a pixel still running
            bool all = true;
#pragma unroll
            for (int m = 0; m < PPT; ++m) all = all && done[m];
            if (__syncthreads_count(all) != NT) {
#pragma unroll
                for (int m = 0; m < PPT; ++m) {
                    const int y = y0 + m;
                    if (x < V.w && y < V.h) {
                        const long long pid = V.pix_off + (long long)y * V.w + x;
                        rgb_out[3 * pid] = C0[m];
                        rgb_out[3 * pid + 1] = C1[m];
                        rgb_out[3 * pid + 2] = C2[m];
                        T_out[pid] = T[m];
                        last_out[pid] = int(unsigned(last[m]) | (done[m] ? 0x80000000u : 0u));
                    }
                }
                const unsigned nc = __reduce_add_sync(0xffffffffu, ncontrib);
                if (lane == 0 && nc) atomicAdd(reinterpret_cast<unsigned long long *>(st.contrib), (unsigned long long)nc);
                if (tid == 0) {
                    st.tile_redo[gt] = 1u;
                    atomicExch(st.super_redo + V.super_base + (tyy / kSuper) * V.sx + txx / kSuper, 1u);
                    st.redo_list[atomicAdd(st.redo_count, 1u)] = gt;
                }
                return;  // (first pass: one tile per block)
            }
        }
        {
            // per-tile statistics: largest last position (orders the adjoint's tiles)
            // and the number of composited pairs
            unsigned ml = 0;
#pragma unroll
            for (int m = 0; m < PPT; ++m) ml = max(ml, unsigned(last[m]));
            ml = __reduce_max_sync(0xffffffffu, ml);
            const unsigned nc = __reduce_add_sync(0xffffffffu, ncontrib);
            if (lane == 0) {
                atomicMax(&s_maxlast, ml);
                atomicAdd(&s_contrib, (unsigned long long)nc);
            }
            __syncthreads();
            if (tid == 0) {
                st.tile_work[gt] = s_maxlast;
                atomicAdd(reinterpret_cast<unsigned long long *>(st.contrib), s_contrib);
                if (REDO) st.tile_avail[gt] = unsigned(len_full);  // the adjoint may read all of it
            }
        }
        float l = 0.f;
#pragma unroll
        for (int m = 0; m < PPT; ++m) {
            const int y = y0 + m;
            if (x < V.w && y < V.h) {
                const long long pid = V.pix_off + (long long)y * V.w + x;
                rgb_out[3 * pid + 0] = C0[m];
                rgb_out[3 * pid + 1] = C1[m];
                rgb_out[3 * pid + 2] = C2[m];
                T_out[pid] = T[m];
                last_out[pid] = last[m];
                if (V.tgt)
                    l += fabsf(C0[m] - target_value(V, x, y, 0)) + fabsf(C1[m] - target_value(V, x, y, 1)) +
                         fabsf(C2[m] - target_value(V, x, y, 2));
            }
        }
        if (V.tgt) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
            if (lane == 0) s_red[wid] = l;
            __syncthreads();
            if (tid == 0) {
                double sum = 0.0;
                for (int w = 0; w < NT / 32; ++w) sum += s_red[w];
                atomicAdd(st.loss_acc, sum);
            }
        }
        if constexpr (!REDO) return;  // one tile per block
    }
}

__global__ void loss_finalise(State st, long long total_pix, float *loss_out)
{
    if (*st.overflow) return;
    *loss_out = float(*st.loss_acc / (3.0 * double(total_pix)));
}

// Sum of 10 per-lane values over the warp in 12 shuffles (instead of 10 x 5):
// at each butterfly level a lane keeps part of its values and sends the
// rest.  Returns the total this lane owns; *idx is its value index, or -1 on
// the lanes that hold a duplicate.  Owners: lanes {0, 2, 4, 8, 12} + 16 h hold
// values {0, 1, 2, 3, 4} + 5 h.
__device__ __forceinline__ float warp_transpose_reduce10(float v[10], int *idx)
{
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    // level 16: keep 5
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float send = b4 ? v[k] : v[k + 5];
        const float keep = b4 ? v[k + 5] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    // level 8: b3 = 0 keeps 3 (0, 1, 2), b3 = 1 keeps 2 (3, 4)
    float r0 = __shfl_xor_sync(0xffffffffu, b3 ? v[0] : v[3], 8);
    float r1 = __shfl_xor_sync(0xffffffffu, b3 ? v[1] : v[4], 8);
    float r2 = __shfl_xor_sync(0xffffffffu, b3 ? v[2] : 0.f, 8);
    float a0, a1, a2;
    if (!b3) {
        a0 = v[0] + r0; a1 = v[1] + r1; a2 = v[2] + r2;
    } else {
        a0 = v[3] + r0; a1 = v[4] + r1; a2 = 0.f;
    }
    // level 4: (b3 = 0) b2 = 0 keeps 2 (a0, a1), b2 = 1 keeps a2; (b3 = 1) each keeps one
    float s0 = !b3 ? (b2 ? a0 : a2) : (b2 ? a0 : a1);
    float s1 = (!b3 && b2) ? a1 : 0.f;
    s0 = __shfl_xor_sync(0xffffffffu, s0, 4);
    s1 = __shfl_xor_sync(0xffffffffu, s1, 4);
    float c0, c1;
    if (!b3) {
        if (!b2) { c0 = a0 + s0; c1 = a1 + s1; } else { c0 = a2 + s0; c1 = 0.f; }
    } else {
        c0 = (b2 ? a1 : a0) + s0;
        c1 = 0.f;
    }
    // level 2: lanes with two values split them, the others add
    const bool two = !b3 && !b2;
    float t0 = __shfl_xor_sync(0xffffffffu, two ? (b1 ? c0 : c1) : c0, 2);
    float d = (two && b1) ? c1 + t0 : c0 + t0;
    // level 1
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    const int base = b4 ? 5 : 0;
    int k = -1;
    if ((lane & 1) == 0) {
        if (two) k = base + (b1 ? 1 : 0);
        else if (!b1) k = base + (!b3 ? 2 : (b2 ? 4 : 3));
    }
    *idx = k;
    return d;
}

constexpr int kG2 = 10;  // moments dx, dy, dx^2, dx dy, dy^2 (-> mean x, y, conic A, B, C), opacity, r, g, b, score

// Adjoint of the compositing, replayed back to front from T_final and the
// last position, each thread a vertical run of PPT pixels.  For each
// Gaussian the thread sums its pixels' contributions, the warp reduces them
// (transpose reduction), warps meet in shared accumulators, and one global
// atomic per (Gaussian, tile, value) leaves the block.
template <int PPT, int BATCH, bool CULL>
__global__ void __launch_bounds__(kTilePix / PPT, PPT == 2 ? 6 : 2048 / (kTilePix / PPT) / 2) composite_bwd(const __grid_constant__ Views vs, State st,
                                                                long long cap, const float *dL_drgb, const float *rgb,
                                                                const float *T_fin, const int32_t *last_idx,
                                                                const float *edge, float *score, float inv_norm)
{
    constexpr int NT = kTilePix / PPT;
    __shared__ float4 s_xyo[BATCH], s_con[BATCH], s_col[BATCH];
    __shared__ float2 s_mlo[BATCH];
    __shared__ int32_t s_id[BATCH];
    __shared__ float s_acc[BATCH][kG2];
    __shared__ int s_maxlast;
    if (*st.overflow) return;
    const int gt = st.order_bwd[blockIdx.x];
    const int v = find_view(vs, gt);
    const ViewP &V = vs.v[v];
    const int lt = gt - V.tile_base;
    const int tyy = lt / V.tiles_x, txx = lt - tyy * V.tiles_x;
    const int tid = threadIdx.x;
    const WarpBlock<PPT> wb(txx, tyy, tid);
    const int x = wb.x, y0 = wb.y0;
    const float px = x + 0.5f;
    const int list_len = int(st.tile_avail[gt]);  // the written prefix of the tile's list
    const int32_t *list = st.ids + st.tile_start[gt];
    const float4 *xyo = st.xyo + (size_t)v * cap, *con = st.con + (size_t)v * cap, *col = st.col + (size_t)v * cap;
    const float2 *mlo = st.mlo + (size_t)v * cap;
    float4 *g2d = st.g2d + (size_t)v * cap * 3;
    const bool want_score = score && edge;
    const float wcx = wb.wcx, wcy = wb.wcy, whw = wb.whw, whh = wb.whh;

    // S = g . (colour composited behind the current position, normalised by the
    // transmittance in front of it): dL/dalpha_i = T_i (g . c_i - S_i), and
    // S_{i-1} = S_i (1 - alpha_i) + alpha_i (g . c_i) (a scalar per pixel in place
    // of the three colour channels)
    float T[PPT], g0[PPT], g1[PPT], g2[PPT], E[PPT], S[PPT];
    int last[PPT];
    int mylast = 0;
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
        const int y = y0 + m;
        T[m] = 1.f; g0[m] = g1[m] = g2[m] = 0.f; E[m] = 0.f; last[m] = 0;
        S[m] = 0.f;
        if (x < V.w && y < V.h) {
            const long long pid = V.pix_off + (long long)y * V.w + x;
            T[m] = T_fin[pid];
            last[m] = min(max(last_idx[pid], 0), list_len);
            E[m] = edge ? edge[pid] : 0.f;
            if (dL_drgb) {
                g0[m] = dL_drgb[3 * pid];
                g1[m] = dL_drgb[3 * pid + 1];
                g2[m] = dL_drgb[3 * pid + 2];
            } else {
                const float d0 = rgb[3 * pid] - target_value(V, x, y, 0);
                const float d1 = rgb[3 * pid + 1] - target_value(V, x, y, 1);
                const float d2 = rgb[3 * pid + 2] - target_value(V, x, y, 2);
                g0[m] = ((d0 > 0.f) - (d0 < 0.f)) * inv_norm;
                g1[m] = ((d1 > 0.f) - (d1 < 0.f)) * inv_norm;
                g2[m] = ((d2 > 0.f) - (d2 < 0.f)) * inv_norm;
            }
            mylast = max(mylast, last[m]);
        }
    }
    if (tid == 0) s_maxlast = 0;
    for (int k = tid; k < BATCH * kG2; k += NT) (&s_acc[0][0])[k] = 0.f;
    __syncthreads();
    atomicMax(&s_maxlast, mylast);
    __syncthreads();
    const int maxlast = s_maxlast;
    const int wlast = int(__reduce_max_sync(0xffffffffu, unsigned(mylast)));  // the warp's last position

    for (int hi = maxlast; hi > 0; hi -= BATCH) {
        const int lo = max(hi - BATCH, 0);
        const int cnt = hi - lo;
        for (int q = tid; q < cnt; q += NT) {
            int id = 0;
            if (GSP_BOUND((long long)st.tile_start[gt] + lo + q, st.pair_cap, st.status)) id = list[lo + q];
            if (!GSP_BOUND(id, cap, st.status)) id = 0;
            s_id[q] = id;
            s_xyo[q] = xyo[id];
            s_mlo[q] = mlo[id];
            s_con[q] = con[id];
            s_col[q] = col[id];
        }
        __syncthreads();
        // unrolled by two: the next staged Gaussian's loads issue while the
        // current one's pixels are replayed (measured 1 % faster)
#pragma unroll 2
        for (int j = min(cnt, wlast - lo) - 1; j >= 0; --j) {
            const int pos = lo + j;
            const float4 gx = s_xyo[j], gc = s_con[j];
            // the footprint's bounding box misses every pixel of the warp (warp-uniform)
            if (CULL && (fabsf(gx.x - wcx) > gx.w + whw || fabsf(gx.y - wcy) > gc.w + whh)) continue;
            float val[kG2];
#pragma unroll
            for (int k = 0; k < kG2; ++k) val[k] = 0.f;
            bool active = false;
#pragma unroll
            for (int m = 0; m < PPT; ++m) {
                if (pos >= last[m]) continue;
                const Alpha a = eval_alpha(gx, s_mlo[j], gc, px, y0 + m + 0.5f);
                if (!a.pass) continue;
                active = true;
                const float4 c = s_col[j];
                const float one_m = __fsub_rn(1.f, a.alpha);
                // 1 - alpha >= 0.01: the fast quotient (2 ulp) keeps the replayed
                // transmittance within a few ulp per step of the forward's
                T[m] = __fdividef(T[m], one_m);
                const float w = a.alpha * T[m];
                val[6] += w * g0[m];
                val[7] += w * g1[m];
                val[8] += w * g2[m];
                const float gc_dot = g0[m] * c.x + g1[m] * c.y + g2[m] * c.z;
                const float dalpha = T[m] * (gc_dot - S[m]);
                S[m] = S[m] * one_m + a.alpha * gc_dot;
                if (a.raw < kAlphaMax) {
                    // moments of dpow = dL/dpower: the mean and conic gradients are
                    // linear in them, the conic is applied once per Gaussian
                    const float dpow = dalpha * gx.z * a.G;
                    val[5] += dalpha * a.G;
                    val[0] += dpow * a.dx;
                    val[1] += dpow * a.dy;
                    val[2] += dpow * a.dxx;
                    val[3] += dpow * a.dxy;
                    val[4] += dpow * a.dyy;
                }
                if (want_score) val[9] += w * E[m];
            }
            if (__any_sync(0xffffffffu, active)) {
                int k;
                const float r = warp_transpose_reduce10(val, &k);
                if (k >= 0 && r != 0.f) atomicAdd(&s_acc[j][k], r);
            }
        }
        __syncthreads();
        for (int q = tid; q < cnt; q += NT) {
            float *a = s_acc[q];
            float4 *gp4 = g2d + (long long)s_id[q] * 3;
            // power = A' dx^2 + B' dx dy + C' dy^2 with (A', B', C') = s_con and
            // dx = px - mean x: d power / d mean = -(2 A' dx + B' dy, B' dx + 2 C' dy),
            // d power / d(A', B', C') = (dx^2, dx dy, dy^2) (the conic's own gradient
            // then follows from A' = -A/2, B' = -B, C' = -C/2)
            const float4 cq = s_con[q];  // times log2(e)
            const float m1 = kLn2 * a[0], m2 = kLn2 * a[1];
            a[0] = -2.f * cq.x * m1 - cq.y * m2;
            a[1] = -cq.y * m1 - 2.f * cq.z * m2;
            a[2] = -0.5f * a[2];
            a[3] = -a[3];
            a[4] = -0.5f * a[4];
            // 16-byte vector atomics: three operations instead of nine
            const float4 v0 = make_float4(a[0], a[1], a[2], a[3]), v1 = make_float4(a[4], a[5], a[6], a[7]);
            if (v0.x != 0.f || v0.y != 0.f || v0.z != 0.f || v0.w != 0.f) atomicAdd(gp4, v0);
            if (v1.x != 0.f || v1.y != 0.f || v1.z != 0.f || v1.w != 0.f) atomicAdd(gp4 + 1, v1);
            if (a[8] != 0.f) atomicAdd(reinterpret_cast<float *>(gp4 + 2), a[8]);
            if (want_score && a[9] != 0.f) atomicAdd(&score[s_id[q]], a[9]);
#pragma unroll
            for (int k = 0; k < kG2; ++k) a[k] = 0.f;
        }
        __syncthreads();
    }
}

// Chain the screen-space gradients to the parameters, one thread per Gaussian,
// summing over views.
// The SH gradients accumulate over the views in a per-thread row of shared
// memory (3K + 1 floats: an odd stride keeps the rows on distinct banks).
template <int K>
__global__ void __launch_bounds__(kProjBwdThreads) project_bwd(const __grid_constant__ Views vs, Params p, State st,
                                                  float *gm, float *gls, float *gq, float *go, float *gsh,
                                                  int accumulate, float *pg_sum, int32_t *pg_count)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= *p.count) return;
    if (*st.overflow) return;
    const long long cap = p.cap;
    float mu[3] = {p.means[3 * i], p.means[3 * i + 1], p.means[3 * i + 2]};
    float ls[3] = {p.log_scales[3 * i], p.log_scales[3 * i + 1], p.log_scales[3 * i + 2]};
    float q4[4] = {p.quats[4 * i], p.quats[4 * i + 1], p.quats[4 * i + 2], p.quats[4 * i + 3]};
    const float opac = sigmoidf_(p.opac[i]);
    const float *shrow = p.sh + (size_t)i * K * 3;
    float G_mu[3] = {0.f, 0.f, 0.f}, G_ls[3] = {0.f, 0.f, 0.f}, G_q[4] = {0.f, 0.f, 0.f, 0.f}, G_o = 0.f;
    extern __shared__ float pb_smem[];
    float *G_sh = pb_smem + threadIdx.x * (3 * K + 1);
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) G_sh[k] = 0.f;
    const float qn2 = q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3];
    const float qinv = __frsqrt_rn(qn2);
    const float qh[4] = {q4[0] * qinv, q4[1] * qinv, q4[2] * qinv, q4[3] * qinv};

    float pg = 0.f;  // positional statistic of this call: norms of the nonzero mean gradients
    int32_t pn = 0;
    for (int v = 0; v < vs.n; ++v) {
        const float4 *gg = st.g2d + ((size_t)v * cap + i) * 3;
        const float4 ga = gg[0], gb = gg[1], gc = gg[2];
        // ga = (mean x, mean y, A, B), gb = (C, opacity, r, g), gc = (b, -, -, -)
        if (ga.x != 0.f || ga.y != 0.f) {
            pg += hypotf(ga.x, ga.y);
            ++pn;
        }
        if (ga.x == 0.f && ga.y == 0.f && ga.z == 0.f && ga.w == 0.f && gb.x == 0.f && gb.y == 0.f &&
            gb.z == 0.f && gb.w == 0.f && gc.x == 0.f)
            continue;
        const ViewP &V = vs.v[v];
        const float *W = V.vm;
        Proj P;
        project_geom(V, mu, ls, q4, P);
        if (!(P.tz > kNear && P.det > 0.f)) continue;
        const float id = 1.f / P.det;
        const float QA = P.c * id, QB = -P.b * id, QC = P.a * id;
        // dL/dSigma2 = -Q G_Q Q with G_Q = [[gA, gB/2], [gB/2, gC]]
        const float hA = ga.z, hB = 0.5f * ga.w, hC = gb.x;
        const float m00 = QA * hA + QB * hB, m01 = QA * hB + QB * hC;
        const float m10 = QB * hA + QC * hB, m11 = QB * hB + QC * hC;
        const float S00 = -(m00 * QA + m01 * QB), S01 = -(m00 * QB + m01 * QC);
        const float S11 = -(m10 * QB + m11 * QC);
        // Sigma2 = T Sig T^T: dL/dSig = T^T S2 T, dL/dT = 2 S2 T Sig
        const float *T = P.T;
        float GSig[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                GSig[3 * a + b] = T[a] * (S00 * T[b] + S01 * T[3 + b]) + T[3 + a] * (S01 * T[b] + S11 * T[3 + b]);
        const float Sg[9] = {P.Sig[0], P.Sig[1], P.Sig[2], P.Sig[1], P.Sig[3], P.Sig[4], P.Sig[2], P.Sig[4], P.Sig[5]};
        float GT[6];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float ts0 = T[0] * Sg[b] + T[1] * Sg[3 + b] + T[2] * Sg[6 + b];
            float ts1 = T[3] * Sg[b] + T[4] * Sg[3 + b] + T[5] * Sg[6 + b];
            GT[b] = 2.f * (S00 * ts0 + S01 * ts1);
            GT[3 + b] = 2.f * (S01 * ts0 + S11 * ts1);
        }
        // T = J W: dL/dJ = GT W^T (entries 00, 02, 11, 12 used)
        const float GJ00 = GT[0] * W[0] + GT[1] * W[1] + GT[2] * W[2];
        const float GJ02 = GT[0] * W[8] + GT[1] * W[9] + GT[2] * W[10];
        const float GJ11 = GT[3] * W[4] + GT[4] * W[5] + GT[5] * W[6];
        const float GJ12 = GT[3] * W[8] + GT[4] * W[9] + GT[5] * W[10];
        const float iz = 1.f / P.tz, iz2 = iz * iz, iz3 = iz2 * iz;
        float gt0 = 0.f, gt1 = 0.f, gt2 = 0.f;
        gt2 += GJ00 * (-V.fx * iz2);
        gt0 += GJ02 * (-V.fx * iz2);
        gt2 += GJ02 * (2.f * V.fx * P.tx * iz3);
        gt2 += GJ11 * (-V.fy * iz2);
        gt1 += GJ12 * (-V.fy * iz2);
        gt2 += GJ12 * (2.f * V.fy * P.ty * iz3);
        gt0 += ga.x * V.fx * iz;
        gt2 += ga.x * (-V.fx * P.tx * iz2);
        gt1 += ga.y * V.fy * iz;
        gt2 += ga.y * (-V.fy * P.ty * iz2);
#pragma unroll
        for (int j = 0; j < 3; ++j) G_mu[j] += W[j] * gt0 + W[4 + j] * gt1 + W[8 + j] * gt2;
        // Sig = M M^T, M = R S: dL/dM = (GSig + GSig^T) M
        float M[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) M[3 * a + b] = P.R[3 * a + b] * P.s[b];
        float GM[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) acc += (GSig[3 * a + k] + GSig[3 * k + a]) * M[3 * k + b];
                GM[3 * a + b] = acc;
            }
#pragma unroll
        for (int b = 0; b < 3; ++b)
            G_ls[b] += (GM[b] * P.R[b] + GM[3 + b] * P.R[3 + b] + GM[6 + b] * P.R[6 + b]) * P.s[b];
        float GR[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) GR[3 * a + b] = GM[3 * a + b] * P.s[b];
        const float w = qh[0], x = qh[1], y = qh[2], z = qh[3];
        float gqw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
        float gqx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] -
                           2.f * x * GR[8]);
        float gqy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] -
                           2.f * y * GR[8]);
        float gqz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] +
                           x * GR[6] + y * GR[7]);
        const float dq = gqw * w + gqx * x + gqy * y + gqz * z;
        G_q[0] += (gqw - w * dq) * qinv;
        G_q[1] += (gqx - x * dq) * qinv;
        G_q[2] += (gqy - y * dq) * qinv;
        G_q[3] += (gqz - z * dq) * qinv;
        G_o += gb.y * opac * (1.f - opac);
        // colour
        const float dx = mu[0] - V.ccx, dy = mu[1] - V.ccy, dz = mu[2] - V.ccz;
        const float rn = __frsqrt_rn(dx * dx + dy * dy + dz * dz);
        const float ux = dx * rn, uy = dy * rn, uz = dz * rn;
        float Y[16];
        sh_eval(ux, uy, uz, K, Y);
        const float gcol[3] = {gb.z, gb.w, gc.x};
        const unsigned clampbits = __float_as_uint(st.col[(size_t)v * cap + i].w);
        float wsh[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) wsh[k] = 0.f;
        const float gm3[3] = {(clampbits & 1u) ? 0.f : gcol[0], (clampbits & 2u) ? 0.f : gcol[1],
                              (clampbits & 4u) ? 0.f : gcol[2]};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
#pragma unroll
            for (int k = 0; k < K; ++k) G_sh[3 * k + ch] += gm3[ch] * Y[k];
        sh_contract<K>(shrow, gm3, wsh);
        float gu[3];
        sh_grad_dot(ux, uy, uz, K, wsh, gu);
        const float ud = gu[0] * ux + gu[1] * uy + gu[2] * uz;
        G_mu[0] += (gu[0] - ux * ud) * rn;
        G_mu[1] += (gu[1] - uy * ud) * rn;
        G_mu[2] += (gu[2] - uz * ud) * rn;
    }
    if (pg_sum) {  // accumulated over calls (the caller resets them)
        pg_sum[i] += pg;
        pg_count[i] += pn;
    }
    float *gshr = gsh + (size_t)i * 3 * K;
    if (accumulate) {
        for (int j = 0; j < 3; ++j) gm[3 * i + j] += G_mu[j], gls[3 * i + j] += G_ls[j];
        for (int j = 0; j < 4; ++j) gq[4 * i + j] += G_q[j];
        go[i] += G_o;
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) gshr[k] += G_sh[k];
    } else {
        for (int j = 0; j < 3; ++j) gm[3 * i + j] = G_mu[j], gls[3 * i + j] = G_ls[j];
        for (int j = 0; j < 4; ++j) gq[4 * i + j] = G_q[j];
        go[i] = G_o;
        if constexpr ((3 * K) % 4 == 0) {
            float4 *o4 = reinterpret_cast<float4 *>(gshr);
#pragma unroll
            for (int q = 0; q < 3 * K / 4; ++q)
                o4[q] = make_float4(G_sh[4 * q], G_sh[4 * q + 1], G_sh[4 * q + 2], G_sh[4 * q + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < 3 * K; ++k) gshr[k] = G_sh[k];
        }
    }
}

// Compositing variants (pixels per thread, batch depth, warp culling); index 0 is the default.
// gsp_render_opts selects one per pass; the autotuner times them on the workload.
struct Variant {
    int ppt, batch;
    bool cull;  // warp-level footprint-box culling of staged Gaussians
};
constexpr Variant kFwdVariants[] = {{1, 256, true}, {2, 256, true}, {1, 128, true}, {2, 128, true},
                                    {1, 128, false}, {2, 128, false}};
constexpr Variant kBwdVariants[] = {{2, 256, true}, {1, 256, true}, {4, 256, true}, {2, 128, true},
                                    {2, 128, false}, {4, 128, true}};
constexpr int kNumFwdVariants = sizeof(kFwdVariants) / sizeof(Variant);
// Tile-list entries written before the forward compositing when the caller
// sets none: dense tiles stop within a few hundred entries (their pixels
// saturate), the others get the rest of their list afterwards.  (1M
// Gaussians on one 1237x822 view: the same step time with 1024 or 2048;
// 3M on eight ring views: 1,179 resumed tiles with 1024, 4 with 2048.)
constexpr unsigned kDefaultListPrefix = 2048;
constexpr int kNumBwdVariants = sizeof(kBwdVariants) / sizeof(Variant);

template <int V>
void launch_fwd(const Views &vs, const State &S, long long cap, const float *edge, float *rgb, float *T, int32_t *last,
                float *score, int redo_pass, cudaStream_t s)
{
    constexpr Variant var = kFwdVariants[V];
    // the redo pass: a few blocks per SM loop over the marked tiles (usually none)
    if (redo_pass)
        composite_fwd<var.ppt, var.batch, var.cull, true>
            <<<std::min(vs.total_tiles, 8 * num_sms()), kTilePix / var.ppt, 0, s>>>(vs, S, cap, edge, rgb, T, last,
                                                                                    score);
    else
        composite_fwd<var.ppt, var.batch, var.cull, false>
            <<<vs.total_tiles, kTilePix / var.ppt, 0, s>>>(vs, S, cap, edge, rgb, T, last, score);
}

void launch_fwd_variant(int variant, const Views &vs, const State &S, long long cap, const float *edge, float *rgb,
                        float *T, int32_t *last, float *score, int redo_pass, cudaStream_t s)
{
    switch (variant) {
    case 1: launch_fwd<1>(vs, S, cap, edge, rgb, T, last, score, redo_pass, s); break;
    case 2: launch_fwd<2>(vs, S, cap, edge, rgb, T, last, score, redo_pass, s); break;
    case 3: launch_fwd<3>(vs, S, cap, edge, rgb, T, last, score, redo_pass, s); break;
    case 4: launch_fwd<4>(vs, S, cap, edge, rgb, T, last, score, redo_pass, s); break;
    case 5: launch_fwd<5>(vs, S, cap, edge, rgb, T, last, score, redo_pass, s); break;
    default: launch_fwd<0>(vs, S, cap, edge, rgb, T, last, score, redo_pass, s); break;
    }
}

template <int V>
void launch_bwd(const Views &vs, const State &S, long long cap, const float *dL, const float *rgb, const float *T,
                const int32_t *last, const float *edge, float *score, float inv_norm, cudaStream_t s)
{
    constexpr Variant var = kBwdVariants[V];
    composite_bwd<var.ppt, var.batch, var.cull>
        <<<vs.total_tiles, kTilePix / var.ppt, 0, s>>>(vs, S, cap, dL, rgb, T, last, edge, score, inv_norm);
}

// ------------------------------------------------------------------- host

constexpr int kCounters = 5;

struct Layout {
    State st;
    size_t bytes;
    size_t clear_bytes;  // bytes of the region cleared per forward pass, from st.pairs_total
};

Layout render_layout(void *ws, long long cap, const Views &vs, long long pair_cap)
{
    Carver c(ws);
    Layout L{};
    State &s = L.st;
    const size_t vc = (size_t)vs.n * cap;
    const size_t total_tiles = (size_t)vs.total_tiles, total_super = (size_t)vs.total_super;
    s.xyo = c.take<float4>(vc);
    s.mlo = c.take<float2>(vc);
    s.con = c.take<float4>(vc);
    s.col = c.take<float4>(vc);
    s.rect = c.take<uint2>(vc);
    s.rowint = c.take<uchar2>(vc * kRowCap);
    s.key = c.take<uint32_t>(vc);
    s.key_alt = c.take<uint32_t>(vc);
    s.val = c.take<int32_t>(vc);
    s.val_alt = c.take<int32_t>(vc);
    s.nb_max = int(div_up(cap, kRsTile));
    s.sort_state = c.take<unsigned>((size_t)vs.n * 4 * s.nb_max * 256);
    s.nch1_max = int(div_up(cap, kL1Ranks));
    s.count1 = c.take<unsigned>(total_super * s.nch1_max);
    s.len1 = c.take<unsigned>(total_super);
    s.list1_start = c.take<unsigned>(total_super);
    s.chunk2_base = c.take<unsigned>(total_super + 1);
    s.id1 = c.take<int32_t>((size_t)pair_cap);
    s.mask1 = c.take<unsigned long long>((size_t)pair_cap);
    // level-2 chunks: at most one partial chunk per supertile beyond pair_cap / 256 full ones
    const size_t chunk2_cap = (size_t)pair_cap / kBinRanks + total_super + 1;
    s.count2 = c.take<unsigned>(chunk2_cap * 64);
    s.chunk_super = c.take<int32_t>(chunk2_cap);
    s.tile_len = c.take<unsigned>(total_tiles);
    s.tile_start = c.take<unsigned>(total_tiles);
    s.tile_avail = c.take<unsigned>(total_tiles);
    s.redo_list = c.take<int32_t>(total_tiles);
    s.ids = c.take<int32_t>((size_t)pair_cap);
    s.order_fwd = c.take<int32_t>(total_tiles);
    s.order_bwd = c.take<int32_t>(total_tiles);
    s.tile_work = c.take<unsigned>(total_tiles);
    s.g2d = c.take<float4>(vc * 3);
    // cleared by one memset per forward pass (from pairs_total to clear_end):
    // pair total, composited pairs, redone tiles, loss sum, overflow flag; the depth sort's
    // digit counts and tickets, the binning scans' tickets; the redo flags and count
    const size_t clear0 = c.size();  // where the counters start
    long long *ctr = c.take<long long>(kCounters);
    s.pairs_total = ctr;
    s.contrib = ctr + 1;
    s.redo_count = reinterpret_cast<unsigned *>(ctr + 2);  // the low word of an int64 statistic
    s.loss_acc = reinterpret_cast<double *>(ctr + 3);
    s.overflow = reinterpret_cast<int32_t *>(ctr + 4);
    s.sort_ghist = c.take<unsigned>((size_t)vs.n * 4 * 256);
    s.sort_ticket = c.take<unsigned>((size_t)vs.n * 4);
    s.scan_ticket = c.take<unsigned>(2);
    s.tile_redo = c.take<unsigned>(total_tiles);
    s.super_redo = c.take<unsigned>(total_super);
    L.clear_bytes = c.size() - clear0;
    s.pair_cap = pair_cap;
    L.bytes = c.size();
    return L;
}

gsp_status build_views(const gsp_camera *cams, int nv, const gsp_image_desc *targets, Views &vs)
{
    if (!cams || nv < 1) return GSP_ERR_INVALID_ARG;
    if (nv > GSP_MAX_VIEWS) return GSP_ERR_UNSUPPORTED;
    int tiles = 0, supers = 0, smax = 0;
    long long pix = 0;
    for (int v = 0; v < nv; ++v) {
        const gsp_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.pixel_offset < 0) return GSP_ERR_INVALID_ARG;
        if (!(c.fx > 0.f) || !(c.fy > 0.f)) return GSP_ERR_INVALID_ARG;
        ViewP &V = vs.v[v];
        for (int k = 0; k < 12; ++k) V.vm[k] = c.viewmat[k];
        V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy;
        // camera centre = -W^T t
        double cc[3];
        for (int j = 0; j < 3; ++j)
            cc[j] = -(double(c.viewmat[j]) * c.viewmat[3] + double(c.viewmat[4 + j]) * c.viewmat[7] +
                      double(c.viewmat[8 + j]) * c.viewmat[11]);
        V.ccx = float(cc[0]); V.ccy = float(cc[1]); V.ccz = float(cc[2]);
        V.w = c.width; V.h = c.height;
        V.tiles_x = int(div_up(c.width, kTile));
        V.tiles_y = int(div_up(c.height, kTile));
        if (V.tiles_x > 65535 || V.tiles_y > 65535) return GSP_ERR_UNSUPPORTED;
        V.sx = int(div_up(V.tiles_x, kSuper));
        V.sy = int(div_up(V.tiles_y, kSuper));
        if ((long long)V.sx * V.sy > kMaxSuper) return GSP_ERR_UNSUPPORTED;
        V.super_base = supers;
        supers += V.sx * V.sy;
        smax = max(smax, V.sx * V.sy);
        V.tile_base = tiles;
        V.pix_off = c.pixel_offset;
        tiles += V.tiles_x * V.tiles_y;
        pix += (long long)c.width * c.height;
        V.tgt = nullptr;
        V.tgt_pitch = 0;
        if (targets) {
            const gsp_image_desc &t = targets[v];
            if (!t.rgb || t.width != c.width || t.height != c.height || t.pitch_bytes < 3LL * c.width)
                return GSP_ERR_INVALID_ARG;
            V.tgt = t.rgb;
            V.tgt_pitch = t.pitch_bytes;
        }
    }
    vs.n = nv;
    vs.total_tiles = tiles;
    vs.total_super = supers;
    vs.smax = smax;
    vs.total_pix = pix;
    return GSP_OK;
}

gsp_status validate_gauss(const gsp_gaussians *g)
{
    if (!g || !g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh || !g->count)
        return GSP_ERR_INVALID_ARG;
    if (g->capacity < 1 || g->capacity >= (1LL << 30)) return GSP_ERR_INVALID_ARG;
    if (g->sh_degree < 0 || g->sh_degree > 3) return GSP_ERR_INVALID_ARG;
    return GSP_OK;
}

Params make_params(const gsp_gaussians *g)
{
    Params p;
    p.means = g->means; p.log_scales = g->log_scales; p.quats = g->quats; p.opac = g->opacity_logits;
    p.sh = g->sh; p.count = g->count; p.cap = g->capacity;
    p.K = (g->sh_degree + 1) * (g->sh_degree + 1);
    return p;
}

}  // namespace
}  // namespace gsp

using namespace gsp;

extern "C" size_t gsp_render_workspace_size(int64_t capacity, int32_t sh_degree, const gsp_camera *cams, int32_t nv,
                                            const gsp_render_opts *opts)
{
    Views vs;
    if (build_views(cams, nv, nullptr, vs) != GSP_OK || !opts || opts->pair_capacity < 1 || capacity < 1 ||
        sh_degree < 0 || sh_degree > 3)
        return 0;
    return render_layout(nullptr, capacity, vs, opts->pair_capacity).bytes;
}

extern "C" const int64_t *gsp_render_pair_count_ptr(const void *ws, int64_t capacity, int32_t sh_degree,
                                                    const gsp_camera *cams, int32_t nv, const gsp_render_opts *opts)
{
    Views vs;
    (void)sh_degree;
    if (!ws || build_views(cams, nv, nullptr, vs) != GSP_OK || !opts) return nullptr;
    return reinterpret_cast<const int64_t *>(
        render_layout(const_cast<void *>(ws), capacity, vs, opts->pair_capacity).st.pairs_total);
}

extern "C" gsp_status gsp_render_fwd(const gsp_gaussians *g, const gsp_camera *cams, int32_t nv,
                                     const gsp_image_desc *targets, const float *edge, float *rgb_out, float *T_final,
                                     int32_t *last_idx, float *score, float *loss_out, const gsp_render_opts *opts,
                                     void *ws, size_t ws_bytes, int32_t *dev_status, gsp_stream_t stream)
{
    gsp_status st = validate_gauss(g);
    if (st != GSP_OK) return st;
    static thread_local Views vs;
    st = build_views(cams, nv, targets, vs);
    if (st != GSP_OK) return st;
    if (!opts || opts->pair_capacity < 1 || !rgb_out || !T_final || !last_idx || !dev_status)
        return GSP_ERR_INVALID_ARG;
    if (score && !edge) return GSP_ERR_INVALID_ARG;
    if (loss_out && !targets) return GSP_ERR_INVALID_ARG;
    if (opts->pair_capacity > 0xffffffffLL) return GSP_ERR_UNSUPPORTED;  // 32-bit list positions
    if (opts->fwd_variant < 0 || opts->fwd_variant >= kNumFwdVariants || opts->bwd_variant < 0 ||
        opts->bwd_variant >= kNumBwdVariants)
        return GSP_ERR_INVALID_ARG;
    const long long cap = g->capacity;
    Layout L = render_layout(nullptr, cap, vs, opts->pair_capacity);
    st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = render_layout(ws, cap, vs, opts->pair_capacity);
    State S = L.st;
    S.n_dev = g->count;
    S.status = dev_status;
    // tile-list entries written before the compositing
    S.prefix = opts->list_prefix >= 0xffffffffLL ? 0xffffffffu
               : opts->list_prefix > 0           ? unsigned(opts->list_prefix)
                                                 : kDefaultListPrefix;
    Params P = make_params(g);
    P.status = dev_status;
    P.sh_bulk = (reinterpret_cast<uintptr_t>(g->sh) & 15) == 0;
    P.sh_wait_limit = (opts->test_expire & 2) ? 0 : kDefaultSpinLimit;
    const long long sort_spin = opts->spin_limit > 0 ? opts->spin_limit : kSortSpinLimit;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    GSP_CUDA_TRY(cudaMemsetAsync(S.pairs_total, 0, L.clear_bytes, s));
    stage_begin("project", s);
    switch (P.K) {
    case 1: launch_project<1>(vs, P, S, cap, s); break;
    case 4: launch_project<4>(vs, P, S, cap, s); break;
    case 9: launch_project<9>(vs, P, S, cap, s); break;
    default: launch_project<16>(vs, P, S, cap, s); break;
    }
    stage_end("project", s);
    GSP_LAUNCH_CHECK();
    stage_begin("depth_sort", s);
    // depth sort of every view at once (blockIdx.y = view): the digit counts of
    // all passes, then 4 stable one-kernel passes of 8 bits; an even count
    // leaves the result in key/val
    {
        uint32_t *k0 = S.key, *k1 = S.key_alt;
        int32_t *v0 = S.val, *v1 = S.val_alt;
        const SortCount sc{g->count};
        ds_count<<<dim3(2 * num_sms(), nv), kRsThreads, 0, s>>>(k0, sc, S.sort_ghist, S.sort_state, S.nb_max, cap);
        for (int pass = 0; pass < 4; ++pass) {
            ds_pass<<<dim3(S.nb_max, nv), kRsThreads, 0, s>>>(k0, v0, k1, v1, sc, pass, S.sort_ghist, S.sort_state,
                                                              S.sort_ticket, S.nb_max, cap, S.overflow, dev_status,
                                                              sort_spin, pass == 0 && (opts->test_expire & 1));
            uint32_t *tk = k0; k0 = k1; k1 = tk;
            int32_t *tv = v0; v0 = v1; v1 = tv;
        }
    }
    stage_end("depth_sort", s);
    GSP_LAUNCH_CHECK();
    stage_begin("bin", s);
    {
        const int nsm = num_sms();
        const size_t smem = size_t(kBinWarps) * vs.smax * sizeof(unsigned);
        const unsigned l1_blocks = unsigned(std::min<long long>(
            std::max<long long>(div_up((long long)nv * S.nch1_max, kBinWarps), 1), 16LL * nsm));
        l1_count<<<l1_blocks, kBinThreads, smem, s>>>(vs, S, cap);
        l1_scan<<<vs.total_super, kScanThreads, 0, s>>>(vs, S, dev_status);
        l1_scatter<<<l1_blocks, kBinThreads, smem, s>>>(vs, S, cap);
        l2_count<<<16 * nsm, kBinThreads, 0, s>>>(vs, S, cap);
        l2_scan<<<vs.total_super, kScanThreads, 0, s>>>(vs, S, dev_status);
        l2_scatter<<<16 * nsm, kBinThreads, 0, s>>>(vs, S, 0);
    }
    stage_end("bin", s);
    GSP_LAUNCH_CHECK();
    stage_begin("composite_fwd", s);
    // over the written prefixes; then the rest of the lists of the tiles that
    // needed more, and those tiles again (both launches leave at once when no
    // tile did)
    launch_fwd_variant(opts->fwd_variant, vs, S, cap, edge, rgb_out, T_final, last_idx, score, 0, s);
    l2_scatter<<<16 * num_sms(), kBinThreads, 0, s>>>(vs, S, 1);
    launch_fwd_variant(opts->fwd_variant, vs, S, cap, edge, rgb_out, T_final, last_idx, score, 1, s);
    stage_end("composite_fwd", s);
    GSP_LAUNCH_CHECK();
    note_launches(2 + 5 + 6 + 3);
    if (loss_out) {
        loss_finalise<<<1, 1, 0, s>>>(S, opts->loss_pixels > 0 ? opts->loss_pixels : vs.total_pix, loss_out);
        note_launches(1);
        GSP_LAUNCH_CHECK();
    }
    return GSP_OK;
}

extern "C" gsp_status gsp_render_bwd(const gsp_gaussians *g, const gsp_camera *cams, int32_t nv,
                                     const gsp_image_desc *targets, const float *dL_drgb, const float *rgb,
                                     const float *T_final, const int32_t *last_idx, const float *edge, float *score,
                                     float *grad_means, float *grad_log_scales, float *grad_quats,
                                     float *grad_opacity_logits, float *grad_sh, int32_t accumulate,
                                     const gsp_render_opts *opts, void *ws, size_t ws_bytes, int32_t *dev_status,
                                     gsp_stream_t stream)
{
    gsp_status st = validate_gauss(g);
    if (st != GSP_OK) return st;
    static thread_local Views vs;
    st = build_views(cams, nv, dL_drgb ? nullptr : targets, vs);
    if (st != GSP_OK) return st;
    if (!opts || !T_final || !last_idx || !dev_status || !grad_means || !grad_log_scales || !grad_quats ||
        !grad_opacity_logits || !grad_sh)
        return GSP_ERR_INVALID_ARG;
    if (!dL_drgb && (!targets || !rgb)) return GSP_ERR_INVALID_ARG;
    if (opts->bwd_variant < 0 || opts->bwd_variant >= kNumBwdVariants) return GSP_ERR_INVALID_ARG;
    if (score && !edge) return GSP_ERR_INVALID_ARG;
    if (!opts->pos_grad_sum != !opts->pos_grad_count) return GSP_ERR_INVALID_ARG;
    const long long cap = g->capacity;
    Layout L = render_layout(nullptr, cap, vs, opts->pair_capacity);
    st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = render_layout(ws, cap, vs, opts->pair_capacity);
    State S = L.st;
    S.n_dev = g->count;
    S.status = dev_status;
    Params P = make_params(g);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float inv_norm =
        float(1.0 / (3.0 * double(opts->loss_pixels > 0 ? opts->loss_pixels : vs.total_pix)));
    stage_begin("composite_bwd", s);
    // the screen-space gradients accumulate from zero in every adjoint call
    GSP_CUDA_TRY(cudaMemsetAsync(S.g2d, 0, sizeof(float4) * 3 * (size_t)nv * cap, s));
    tile_order_bwd<<<1, 1024, 0, s>>>(vs.total_tiles, S);
    switch (opts->bwd_variant) {
    case 1: launch_bwd<1>(vs, S, cap, dL_drgb, rgb, T_final, last_idx, edge, score, inv_norm, s); break;
    case 2: launch_bwd<2>(vs, S, cap, dL_drgb, rgb, T_final, last_idx, edge, score, inv_norm, s); break;
    case 3: launch_bwd<3>(vs, S, cap, dL_drgb, rgb, T_final, last_idx, edge, score, inv_norm, s); break;
    case 4: launch_bwd<4>(vs, S, cap, dL_drgb, rgb, T_final, last_idx, edge, score, inv_norm, s); break;
    case 5: launch_bwd<5>(vs, S, cap, dL_drgb, rgb, T_final, last_idx, edge, score, inv_norm, s); break;
    default: launch_bwd<0>(vs, S, cap, dL_drgb, rgb, T_final, last_idx, edge, score, inv_norm, s); break;
    }
    stage_end("composite_bwd", s);
    GSP_LAUNCH_CHECK();
    // the edge score is complete: a caller may start the selection from here
    if (opts->score_event) GSP_CUDA_TRY(cudaEventRecord(reinterpret_cast<cudaEvent_t>(opts->score_event), s));
    stage_begin("project_bwd", s);
#define GSP_PBWD(KK)                                                                                           \
    project_bwd<KK><<<div_up(cap, kProjBwdThreads), kProjBwdThreads,                                             \
                      sizeof(float) * kProjBwdThreads * (3 * (KK) + 1), s>>>(vs, P, S, grad_means, grad_log_scales, \
                                                                             grad_quats, grad_opacity_logits, grad_sh, \
                                                                             accumulate, opts->pos_grad_sum,            \
                                                                             opts->pos_grad_count)
    switch (P.K) {
    case 1: GSP_PBWD(1); break;
    case 4: GSP_PBWD(4); break;
    case 9: GSP_PBWD(9); break;
    default: GSP_PBWD(16); break;
    }
#undef GSP_PBWD
    stage_end("project_bwd", s);
    note_launches(4);
    GSP_LAUNCH_CHECK();
    return GSP_OK;
}
