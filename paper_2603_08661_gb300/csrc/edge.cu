// Edge-importance map (paper Sec. 2.1): grayscale, 5x5 Gaussian blur, Sobel,
// NMS along the quantised gradient, lower-median normalisation.
//
// Arithmetic.  The luma is formed as the exact integer I = 299 R + 587 G + 114 B
// (= 255000 x the [0, 1] luma).  Blur and Sobel are linear and act on the
// clamp-extended image, so they commute: the Sobel differences are taken first
// on the exact integers (|S| < 2^21, exact in FP32) and the 5x5 blur is applied
// to them in FP32: horizontally with its symmetric taps paired (the pair sums
// of integers are exact), vertically as one FMA chain from the top row down.
// NMS compares squared magnitudes M^2 = gx^2 + gy^2 (the
// comparisons of M and of M^2 agree except at FP32 near-ties), and only kept
// pixels take a square root.  Magnitudes stay in units of 255000 x luma; E =
// M / median is unit-free.
//
// Median.  The lower median of the kept magnitudes is the square root of the
// lower median of the kept M^2 (the square root preserves order), selected
// exactly from the float bit patterns (positive floats order like their bits):
// a 4096-bin histogram of bits [30:19], then the values falling into the
// median's bin are gathered and resolved on bits [18:9] and [8:0].
//
// Fused mode runs every stage of every view in one cooperative launch.  Two
// kernels implement it, the same arithmetic in different schedules; the host
// picks the walk kernel for large batches (less per-pixel overhead) and the
// tile kernel for small ones (more parallelism per pixel row).
//
// Tile kernel (edge_tile_kernel): blocks take 64 x 16 output tiles.
//   A  the tile's RGB halo box is staged in shared memory by a 2-D TMA copy
//      (double-buffered; views whose base or pitch is not 16-byte aligned are
//      read directly), stencil chain in shared memory, NMS, M^2_thin written to
//      E_out, per-view histogram of bits [30:19]
//   then B0, B, C as below, streaming M^2_thin from E_out; D divides in place.
//
// Walk kernel (edge_walk_kernel): four blocks of 4 warps per SM.  The unit of
// work is a warp item: 120 output columns over a band of rows of one view.
//   A  lane L walks the 4 columns xg - 4 + 4 L .. + 3 down the band (lanes 0
//      and 31 hold the halo columns on either side): it loads its pixels'
//      bytes one row ahead, forms their luma, the vertical Sobel parts from
//      the last three luma rows, takes the neighbours' edge columns by warp
//      shuffles for the horizontal Sobel parts and the horizontal blur (both
//      gradient components in one packed FP32x2 operation), advances four
//      partial vertical-blur chains in registers, and decides NMS from the
//      last three M^2 rows (their ring columns by shuffles) and the previous
//      row's direction class (4 bits per column).  Kept M^2
//      values are compacted per row pair into the item's slot, with a keep
//      byte per lane and pair, and counted in a warp histogram of bits
//      [30:19] (two 16-bit counts a word, flushed before they can overflow).
//   -- grid barrier --
//   B0 block v finds view v's median bin of bits [30:19]
//   -- grid barrier --
//   B  every warp streams its items' kept values, collects those in the
//      median bin and counts them on bits [18:9], and appends them to the
//      view's candidate list with one reservation per buffer
//   -- grid barrier --
//   C  block v resolves view v's median: the bin of bits [18:9] from that
//      count, bits [8:0] from one pass over the candidates in it
//   -- grid barrier --
//   D  every warp re-walks its items in chunks of row pairs: the chunk's keep
//      bytes come in at once, its kept values arrive in shared memory by
//      cp.async (all in flight together) and are converted to E =
//      sqrt(M^2) / median by all lanes together, and each E row (zeros and
//      those values) is staged in shared memory for contiguous stores.
// Plain mode launches one kernel per stage and per view, with every
// intermediate in global memory (the unfused reference path); both modes
// perform the same FP32 operations and agree bit for bit.

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace gsp {
namespace {

constexpr int NT = 256;                  // threads of a tile-kernel block (8 warps)
constexpr int kBins1 = 4096, kShift1 = 19;
constexpr int kBins2 = 1024, kShift2 = 9;
constexpr int kBins3 = 512;
constexpr float kTan22 = 0.41421356237309503f;  // tan(22.5 deg) = sqrt(2) - 1

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// Exact integer to float for |i| < 2^22: place i in the mantissa of 1.5 * 2^23
// and subtract (two full-rate operations instead of a conversion).
__device__ __forceinline__ float i2f_exact(int i)
{
    return __fsub_rn(__int_as_float(i + 0x4B400000), 12582912.0f);
}

// The luma 299 R + 587 G + 114 B of a pixel whose bytes are the low three of
// px (R, G, B, any), as an exact float: 256 (R + 2 G) + (43 R + 75 G + 114 B),
// two byte dot products whose weights fit in 8 bits.
__device__ __forceinline__ float luma_exact(unsigned px)
{
    return i2f_exact(int(__dp4a(px, 0x00724B2Bu, __dp4a(px, 0x00000201u, 0u) << 8)));
}

// Vertical 5-tap blur of one column, rows h0 (top) .. h4: the chain
// w2 h0 (+) w1 h1 (+) w0 h2 (+) w1 h3 (+) w2 h4, each step one rounding (the
// walk kernel advances the same chains in place as rows arrive).
__device__ __forceinline__ float vblur5(float h0, float h1, float h2, float h3, float h4, float w0, float w1,
                                        float w2)
{
    return __fmaf_rn(w2, h4, __fmaf_rn(w1, h3, __fmaf_rn(w0, h2, __fmaf_rn(w1, h1, __fmul_rn(w2, h0)))));
}

// Exclusive warp scan of one value per lane; returns the warp total.
__device__ __forceinline__ unsigned warp_exclusive_scan(unsigned x, unsigned *excl)
{
    const int lane = threadIdx.x & 31;
    unsigned inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    *excl = inc - x;
    return __shfl_sync(0xffffffffu, inc, 31);
}

// Exclusive block scan of one value per thread (BT threads); returns the total.
template <int BT = NT>
__device__ unsigned block_exclusive_scan(unsigned x, unsigned *out)
{
    __shared__ unsigned warp_tot[BT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    unsigned base = 0, total = 0;
    for (int w = 0; w < BT / 32; ++w) {
        if (w < wid) base += warp_tot[w];
        total += warp_tot[w];
    }
    *out = base + inc - x;
    __syncthreads();
    return total;
}

// Find the bin of the element of ascending rank `rank` in a histogram (any
// address space; nbins a multiple of BT).  Every thread receives (bin, count
// below the bin).
template <int BT = NT>
__device__ void block_find_bin(const unsigned *hist, int nbins, unsigned rank, int *bin_out,
                               unsigned *below_out)
{
    __shared__ int s_bin;
    __shared__ unsigned s_below;
    const int per = nbins / BT;
    unsigned seg = 0;
    for (int k = 0; k < per; ++k) seg += hist[threadIdx.x * per + k];
    unsigned before;
    block_exclusive_scan<BT>(seg, &before);
    if (rank >= before && rank < before + seg) {
        unsigned acc = before;
        for (int k = 0; k < per; ++k) {
            unsigned h = hist[threadIdx.x * per + k];
            if (rank < acc + h) {
                s_bin = threadIdx.x * per + k;
                s_below = acc;
                break;
            }
            acc += h;
        }
    }
    __syncthreads();
    *bin_out = s_bin;
    *below_out = s_below;
    __syncthreads();
}

// ================================================================ tile kernel

constexpr int TW = 64, TH = 16;  // tile kernel: output tile of 64 x 16 pixels, NT threads
constexpr int IW = TW + 8, IH = TH + 8;  // integer luma with a 4-pixel halo
constexpr int HW = TW + 2, HH = TH + 6;  // after the horizontal blur
constexpr int MW = TW + 2, MH = TH + 2;  // magnitude with a 1-pixel ring

struct TileView {
    const uint8_t *rgb;
    long long pitch;
    long long out_off;
    int w, h;
    int tiles_x;
    int tile_base;
    int ntiles;
    int tma;  // 1: the view's halo tiles are staged by TMA (16-byte aligned base and pitch)
};

// TMA box of one tile's input: the RGB bytes of its halo (TW + 8 pixels plus
// the alignment slack: the box starts 16 bytes before the tile's first pixel,
// a 16-byte boundary since TW * 3 is a multiple of 16) x (TH + 8) rows.
constexpr int kBoxW = 224, kBoxH = TH + 8;
constexpr int kBoxLead = 16;  // bytes between the box start and pixel x0 - 0
static_assert(3 * (TW + 4) + kBoxLead <= kBoxW && (3 * TW) % 16 == 0 && kBoxW % 16 == 0, "TMA box");
static_assert(kBoxLead >= 3 * 4, "the box reaches the left halo");

struct TileArgs {
    TileView v[GSP_MAX_VIEWS];
    int nviews;
    int total_tiles;
    float w0, w1, w2;  // blur taps: centre, +-1, +-2
    float *E;
    uint8_t *mask;
    float *median_out;
    unsigned *hist1;       // [V][kBins1]
    unsigned *hist2;       // [V][kBins2] bits [18:9] of the candidates
    unsigned *sel;         // [V][4]: kept count, median bin of bits [30:19], count below that bin
    unsigned *cand_count;  // [V]
    float *cand;           // candidate values, laid out like E
    unsigned *med_bits;    // [V]
    unsigned *bar;         // grid barrier state [2]
    int32_t *status;
    long long spin_limit;  // grid-barrier polls
    int expire;            // test hook bits: 1 withholds the first grid barrier, 2 makes box waits give up at once
    CUtensorMap tmap[GSP_MAX_VIEWS];  // uint8 [h][3w] with row pitch, box kBoxW x kBoxH
};

// Stage buffers of one tile.  Sobel and the horizontal blur run fused in
// registers (no Sobel buffer); the integer luma I is dead once the blur rows
// exist, so M / Gx / Gy reuse its storage.
struct TileSmem {
    union {
        alignas(16) int I[IH][IW];
        struct {
            float M[MH][MW];
            float Gx[TH][TW], Gy[TH][TW];
        };
    };
    float Hx[HH][HW], Hy[HH][HW];
};

// Staged RGB boxes (two, for the next tile's copy to overlap this tile) and
// their barriers.
struct StageSmem {
    alignas(128) uint8_t box[2][kBoxH][kBoxW];
    unsigned long long bar[2];
};


// Stencil chain for one 64x16 output tile at (x0, y0) of view V.  box: the
// tile's staged RGB bytes (rows y0 - 4 .., bytes from 3 x0 - kBoxLead), or
// null to read the image directly.  Clamp-to-edge indexes the box (or the
// image) at clamped coordinates; the box holds every clamped pixel.
//   luma   I (exact integers), 4 pixels per thread from three 32-bit words of
//          the box where no clamping is needed
//   sobel + horizontal blur, fused: a thread takes a row run of 6 outputs,
//          forms the 10 exact integer Sobel pairs it needs in registers and
//          blurs them (taps paired, same operation order as a plain pass)
//   vertical blur + magnitude: a thread takes a column run of 6 outputs
constexpr int kSegH = 6;                 // row run of the fused Sobel + horizontal blur
constexpr int kSegV = 6;                 // column run of the vertical blur
static_assert(HW % kSegH == 0 && MH % kSegV == 0, "segment runs");
static_assert((HW / kSegH) * HH <= NT && (MH / kSegV) * MW <= NT, "one run per thread");

__device__ void tile_stencil(const TileView &V, int x0, int y0, float w0, float w1, float w2,
                             const uint8_t (*box)[kBoxW], TileSmem &s)
{
    const int tid = threadIdx.x;
    const bool interior = box && x0 >= 4 && x0 + TW + 4 <= V.w && y0 >= 4 && y0 + TH + 4 <= V.h;
    if (interior) {
        // 4 pixels from 12 bytes at box byte 3 c + 4 (c a multiple of 4: word aligned)
        for (int g = tid; g < IH * (IW / 4); g += NT) {
            const int r = g / (IW / 4), c = 4 * (g - r * (IW / 4));
            const unsigned *w = reinterpret_cast<const unsigned *>(&box[r][3 * c + kBoxLead - 12]);
            const unsigned a0 = w[0], a1 = w[1], a2 = w[2];
            const int b0 = a0 & 255, b1 = (a0 >> 8) & 255, b2 = (a0 >> 16) & 255, b3 = a0 >> 24;
            const int b4 = a1 & 255, b5 = (a1 >> 8) & 255, b6 = (a1 >> 16) & 255, b7 = a1 >> 24;
            const int b8 = a2 & 255, b9 = (a2 >> 8) & 255, b10 = (a2 >> 16) & 255, b11 = a2 >> 24;
            *reinterpret_cast<int4 *>(&s.I[r][c]) =
                make_int4(299 * b0 + 587 * b1 + 114 * b2, 299 * b3 + 587 * b4 + 114 * b5,
                          299 * b6 + 587 * b7 + 114 * b8, 299 * b9 + 587 * b10 + 114 * b11);
        }
    } else {
        for (int idx = tid; idx < IH * IW; idx += NT) {
            int r = idx / IW, c = idx - r * IW;
            int yy = clampi(y0 - 4 + r, 0, V.h - 1), xx = clampi(x0 - 4 + c, 0, V.w - 1);
            const uint8_t *p = box ? &box[yy - (y0 - 4)][3 * (xx - x0) + kBoxLead]
                                   : V.rgb + (long long)yy * V.pitch + 3 * xx;
            s.I[r][c] = 299 * int(p[0]) + 587 * int(p[1]) + 114 * int(p[2]);
        }
    }
    __syncthreads();
    // Sobel (exact integers) + horizontal blur: outputs H[r][c0 .. c0 + 5] use
    // Sobel columns c0 .. c0 + 9, which use I rows r .. r + 2, columns c0 .. c0 + 11
    if (tid < (HW / kSegH) * HH) {
        const int r = tid / (HW / kSegH), c0 = kSegH * (tid - r * (HW / kSegH));
        int i0[kSegH + 6], i1[kSegH + 6], i2[kSegH + 6];
#pragma unroll
        for (int j = 0; j < kSegH + 6; j += 2) {
            const int2 u0 = *reinterpret_cast<const int2 *>(&s.I[r][c0 + j]);
            const int2 u1 = *reinterpret_cast<const int2 *>(&s.I[r + 1][c0 + j]);
            const int2 u2 = *reinterpret_cast<const int2 *>(&s.I[r + 2][c0 + j]);
            i0[j] = u0.x; i0[j + 1] = u0.y;
            i1[j] = u1.x; i1[j + 1] = u1.y;
            i2[j] = u2.x; i2[j + 1] = u2.y;
        }
        float fx[kSegH + 4], fy[kSegH + 4];
#pragma unroll
        for (int j = 0; j < kSegH + 4; ++j) {
            const int sx = (i0[j + 2] - i0[j]) + 2 * (i1[j + 2] - i1[j]) + (i2[j + 2] - i2[j]);
            const int sy = (i2[j] - i0[j]) + 2 * (i2[j + 1] - i0[j + 1]) + (i2[j + 2] - i0[j + 2]);
            fx[j] = float(sx);
            fy[j] = float(sy);
        }
#pragma unroll
        for (int j = 0; j < kSegH; ++j) {
            const float ax1 = fx[j + 1] + fx[j + 3], ax2 = fx[j] + fx[j + 4];
            const float ay1 = fy[j + 1] + fy[j + 3], ay2 = fy[j] + fy[j + 4];
            s.Hx[r][c0 + j] = __fmaf_rn(w2, ax2, __fmaf_rn(w1, ax1, __fmul_rn(w0, fx[j + 2])));
            s.Hy[r][c0 + j] = __fmaf_rn(w2, ay2, __fmaf_rn(w1, ay1, __fmul_rn(w0, fy[j + 2])));
        }
    }
    __syncthreads();
    // vertical blur + magnitude: outputs M[r0 .. r0 + 5][c] use H rows r0 .. r0 + 9
    if (tid < (MH / kSegV) * MW) {
        const int seg = tid / MW, c = tid - seg * MW, r0 = kSegV * seg;
        float hx[kSegV + 4], hy[kSegV + 4];
#pragma unroll
        for (int j = 0; j < kSegV + 4; ++j) {
            hx[j] = s.Hx[r0 + j][c];
            hy[j] = s.Hy[r0 + j][c];
        }
        const int xx = x0 - 1 + c;
#pragma unroll
        for (int j = 0; j < kSegV; ++j) {
            const int r = r0 + j;
            const float gx = vblur5(hx[j], hx[j + 1], hx[j + 2], hx[j + 3], hx[j + 4], w0, w1, w2);
            const float gy = vblur5(hy[j], hy[j + 1], hy[j + 2], hy[j + 3], hy[j + 4], w0, w1, w2);
            const int yy = y0 - 1 + r;
            const bool inside = yy >= 0 && yy < V.h && xx >= 0 && xx < V.w;
            s.M[r][c] = inside ? __fmaf_rn(gx, gx, __fmul_rn(gy, gy)) : 0.0f;  // squared magnitude
            if (r >= 1 && r <= TH && c >= 1 && c <= TW) {
                s.Gx[r - 1][c - 1] = gx;
                s.Gy[r - 1][c - 1] = gy;
            }
        }
    }
    __syncthreads();
}

// NMS decision for inner pixel (r, c) of the tile (Sec. 2.1 step 3).
__device__ __forceinline__ float nms_value(const TileSmem &s, int r, int c)
{
    float m = s.M[r + 1][c + 1];
    float gx = s.Gx[r][c], gy = s.Gy[r][c];
    float ax = fabsf(gx), ay = fabsf(gy);
    bool horiz = ay <= __fmul_rn(kTan22, ax);
    bool vert = !horiz && ax <= __fmul_rn(kTan22, ay);
    int sx = vert ? 0 : (gx > 0.f) - (gx < 0.f);
    int sy = horiz ? 0 : (gy > 0.f) - (gy < 0.f);
    float mp = s.M[r + 1 + sy][c + 1 + sx];
    float mm = s.M[r + 1 - sy][c + 1 - sx];
    bool keep = m > 0.f && m >= mp && m > mm;
    return keep ? m : 0.f;
}

__device__ __forceinline__ int tile_view(const TileArgs &a, int tile)
{
    int v = 0;
    while (v + 1 < a.nviews && a.v[v + 1].tile_base <= tile) ++v;
    return v;
}



// 2-D tiled TMA load of one box into shared memory, completed on bar.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tile_origin(const TileArgs &a, int t, int &v, int &x0, int &y0)
{
    v = tile_view(a, t);
    const TileView &V = a.v[v];
    const int lt = t - V.tile_base;
    const int ty = lt / V.tiles_x, tx = lt - ty * V.tiles_x;
    x0 = tx * TW;
    y0 = ty * TH;
}

// Thread 0: stage tile t's RGB box into buffer buf (views without TMA are read directly).
__device__ __forceinline__ void issue_box(const TileArgs &a, StageSmem &stg, int t, int buf)
{
    int v, x0, y0;
    tile_origin(a, t, v, x0, y0);
    if (!a.v[v].tma) return;
    // the previous reads of this buffer (generic proxy) precede the async copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&stg.bar[buf], unsigned(kBoxW * kBoxH));
    tma_load_2d(&stg.box[buf][0][0], &a.tmap[v], 3 * x0 - kBoxLead, y0 - 4, &stg.bar[buf]);
}

__global__ void __launch_bounds__(NT) edge_tile_kernel(const __grid_constant__ TileArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations need 128-byte alignment: the launch adds 128 bytes of slack
    unsigned char *smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    StageSmem &stg = *reinterpret_cast<StageSmem *>(smem_raw);
    TileSmem &s = *reinterpret_cast<TileSmem *>(smem_raw + sizeof(StageSmem));
    unsigned *hist_s = reinterpret_cast<unsigned *>(smem_raw + sizeof(StageSmem) + sizeof(TileSmem));
    const int tid = threadIdx.x;
    const int G = gridDim.x;
    const int t_begin = int((long long)a.total_tiles * blockIdx.x / G);
    const int t_end = int((long long)a.total_tiles * (blockIdx.x + 1) / G);
    const float scale = 1.0f / 255000.0f;

    // ---- phase A: stencil, NMS, M_thin -> E, histogram of bits [30:19]
    // The next tile's box is copied by TMA while this tile is computed.
    if (tid == 0) {
        mbar_init(&stg.bar[0], 1);
        mbar_init(&stg.bar[1], 1);
    }
    __syncthreads();
    if (tid == 0 && t_begin < t_end) issue_box(a, stg, t_begin, 0);
    unsigned uses[2] = {0u, 0u};  // completed phases of each buffer's barrier (block-uniform)
    // The waits for this block's own box copies are bounded by the default limit
    // (a copy that never lands is a fault, not a state to wait out); the hook
    // (expire bit 1) makes them give up at once.  Either way a block that gives
    // up first lets every copy it has in flight land, then leaves.
    const long long box_limit = (a.expire & 2) ? 0 : kDefaultSpinLimit;
    int cur_view = -1;
    for (int t = t_begin, it = 0; t < t_end; ++t, ++it) {
        const int buf = it & 1;
        if (tid == 0 && t + 1 < t_end) issue_box(a, stg, t + 1, buf ^ 1);
        int v, x0, y0;
        tile_origin(a, t, v, x0, y0);
        const TileView &V = a.v[v];
        if (v != cur_view) {
            if (cur_view >= 0) {
                __syncthreads();
                for (int i = tid; i < kBins1; i += NT)
                    if (hist_s[i]) atomicAdd(&a.hist1[(size_t)cur_view * kBins1 + i], hist_s[i]);
            }
            __syncthreads();
            for (int i = tid; i < kBins1; i += NT) hist_s[i] = 0;
            cur_view = v;
        }
        if (V.tma) {
            const bool mine = mbar_wait(&stg.bar[buf], uses[buf] & 1u, box_limit);
            if (!__syncthreads_and(mine)) {
                set_status(a.status, GSP_ERR_TIMEOUT);
                // drain: this tile's copy, and the next tile's if one was issued
                if (tid == 0) {
                    mbar_wait(&stg.bar[buf], uses[buf] & 1u, kDefaultSpinLimit);
                    if (t + 1 < t_end) {
                        int v1, x1, y1;
                        tile_origin(a, t + 1, v1, x1, y1);
                        if (a.v[v1].tma) mbar_wait(&stg.bar[buf ^ 1], uses[buf ^ 1] & 1u, kDefaultSpinLimit);
                    }
                }
                __syncthreads();
                return;
            }
            ++uses[buf];
        }
        tile_stencil(V, x0, y0, a.w0, a.w1, a.w2, V.tma ? stg.box[buf] : nullptr, s);
        for (int idx = tid; idx < TH * TW; idx += NT) {
            int r = idx / TW, c = idx - r * TW;
            int y = y0 + r, x = x0 + c;
            if (y < V.h && x < V.w) {
                float mt = nms_value(s, r, c);
                long long o = V.out_off + (long long)y * V.w + x;
                a.E[o] = mt;
                if (a.mask) a.mask[o] = mt > 0.f;
                if (mt > 0.f) atomicAdd(&hist_s[__float_as_uint(mt) >> kShift1], 1u);
            }
        }
        __syncthreads();
    }
    if (cur_view >= 0) {
        __syncthreads();
        for (int i = tid; i < kBins1; i += NT)
            if (hist_s[i]) atomicAdd(&a.hist1[(size_t)cur_view * kBins1 + i], hist_s[i]);
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status, (a.expire & 1) != 0)) return;

    // ---- phase B0: each view's median bin of bits [30:19] and kept count (block v)
    for (int v = blockIdx.x; v < a.nviews; v += G) {
        const unsigned *h = a.hist1 + (size_t)v * kBins1;
        unsigned seg = 0;
        for (int k = 0; k < kBins1 / NT; ++k) seg += h[tid * (kBins1 / NT) + k];
        unsigned before;
        const unsigned n = block_exclusive_scan(seg, &before);
        int b1 = 0;
        unsigned below = 0;
        if (n > 0) block_find_bin(h, kBins1, (n - 1) / 2, &b1, &below);
        if (tid == 0) {
            a.sel[4 * v + 0] = n;
            a.sel[4 * v + 1] = unsigned(b1);
            a.sel[4 * v + 2] = below;
        }
        __syncthreads();
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status)) return;

    // ---- phase B: stream every view's slice of M_thin (8 loads in flight per
    // thread); the candidates (kept values in the median bin) are compacted per
    // block round, appended with one reservation, and counted on bits [18:9]
    float *cbuf = reinterpret_cast<float *>(&s);  // NT * kStream floats (the stencil buffers are free)
    constexpr int kStream = 8;
    static_assert(sizeof(TileSmem) >= NT * kStream * sizeof(float), "candidate buffer");
    __shared__ unsigned s_base;
    for (int v = 0; v < a.nviews; ++v) {
        const unsigned n = a.sel[4 * v + 0];
        if (n == 0) continue;
        const unsigned b1 = a.sel[4 * v + 1];
        const TileView &V = a.v[v];
        const long long npx = (long long)V.w * V.h;
        const long long lo = npx * blockIdx.x / G, hi = npx * (blockIdx.x + 1) / G;
        const float *src = a.E + V.out_off;
        unsigned *h2 = a.hist2 + (size_t)v * kBins2;
        for (long long base = lo; base < hi; base += NT * kStream) {
            float val[kStream];
            unsigned mine = 0;
#pragma unroll
            for (int k = 0; k < kStream; ++k) {
                const long long e = base + k * NT + tid;
                val[k] = e < hi ? src[e] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < kStream; ++k) {
                const bool pick = val[k] > 0.f && (__float_as_uint(val[k]) >> kShift1) == b1;
                if (!pick) val[k] = -1.f;
                mine += pick;
            }
            unsigned off;
            const unsigned total = block_exclusive_scan(mine, &off);
            if (total == 0) continue;
#pragma unroll
            for (int k = 0; k < kStream; ++k)
                if (val[k] >= 0.f) {
                    cbuf[off++] = val[k];
                    atomicAdd(&h2[(__float_as_uint(val[k]) >> kShift2) & (kBins2 - 1)], 1u);
                }
            if (tid == 0) s_base = atomicAdd(a.cand_count + v, total);
            __syncthreads();
            float *dst = a.cand + V.out_off + s_base;
            for (unsigned i = tid; i < total; i += NT)
                if (GSP_BOUND(s_base + i, (long long)V.w * V.h, a.status)) dst[i] = cbuf[i];
            __syncthreads();
        }
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status)) return;

    // ---- phase C: exact median of each view (block v): the level-2 bin from
    // the candidates' histogram, then bits [8:0] among the candidates in it
    for (int v = blockIdx.x; v < a.nviews; v += G) {
        const unsigned n = a.sel[4 * v + 0];
        unsigned bits = 0;
        if (n > 0) {
            const unsigned b1 = a.sel[4 * v + 1];
            unsigned rank = (n - 1) / 2 - a.sel[4 * v + 2];
            int b2;
            unsigned below2;
            block_find_bin(a.hist2 + (size_t)v * kBins2, kBins2, rank, &b2, &below2);
            rank -= below2;
            for (int i = tid; i < kBins3; i += NT) hist_s[i] = 0;
            __syncthreads();
            const float *cand = a.cand + a.v[v].out_off;
            const unsigned count = a.cand_count[v];
            for (unsigned i = tid; i < count; i += NT) {
                const unsigned cb = __float_as_uint(cand[i]);
                if (((cb >> kShift2) & (kBins2 - 1)) == unsigned(b2)) atomicAdd(&hist_s[cb & (kBins3 - 1)], 1u);
            }
            __syncthreads();
            int b3;
            unsigned below3;
            block_find_bin(hist_s, kBins3, rank, &b3, &below3);
            bits = (b1 << kShift1) | (unsigned(b2) << kShift2) | unsigned(b3);
        }
        if (tid == 0) {
            a.med_bits[v] = bits;
            a.median_out[v] = __fsqrt_rn(__uint_as_float(bits)) * scale;
        }
        __syncthreads();
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status)) return;

    // ---- phase D: E = sqrt(M^2_thin) / median, streaming every view's slice
    for (int v = 0; v < a.nviews; ++v) {
        const float med2 = __uint_as_float(a.med_bits[v]);
        if (!(med2 > 0.f)) continue;
        const float med = __fsqrt_rn(med2);
        const TileView &V = a.v[v];
        const long long npx = (long long)V.w * V.h;
        const long long lo = npx * blockIdx.x / G, hi = npx * (blockIdx.x + 1) / G;
        float *e = a.E + V.out_off;
        for (long long base = lo; base < hi; base += NT * kStream) {
            float val[kStream];
#pragma unroll
            for (int k = 0; k < kStream; ++k) {
                const long long i = base + k * NT + tid;
                val[k] = i < hi ? e[i] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < kStream; ++k) {
                const long long i = base + k * NT + tid;
                if (i < hi && val[k] > 0.f) e[i] = __fdiv_rn(__fsqrt_rn(val[k]), med);
            }
        }
    }
}


// ================================================================ walk kernel
//
// A warp item is 128 image columns over a band of rb rows: lane L holds the 4
// columns cx = xg - 4 + 4 L .. cx + 3; lanes 1..30 produce the item's 120
// output columns xg .. xg + 119 and lanes 0 and 31 compute the 4-column halo
// on either side.  Values a lane needs from its neighbours' columns (Sobel and
// blur halos, the NMS ring) come by warp shuffles.
constexpr int WNT = 128;                      // threads of a walk block (4 warps)
constexpr int kWWarps = WNT / 32;
constexpr int kWalkBlocksPerSM = 4;           // resident walk blocks per SM the plan assumes
constexpr int kQ = 4;                         // columns per lane
constexpr int kItemCols = 32 * kQ - 2 * kQ;   // 120 output columns per item
constexpr int kDPairs = 4;                    // row pairs per phase-D chunk (two chunks staged at once)
constexpr int kBCand = 512;                   // phase-B candidate buffer per warp
constexpr unsigned kFull = 0xffffffffu;

struct EdgeView {
    const uint8_t *rgb;
    long long pitch;
    long long out_off;
    int w, h;
    int groups;     // warp items across the width (120 columns each)
    int bands;      // warp items down the height
    int item_base;  // first item of the view
};

struct EdgeArgs {
    EdgeView v[GSP_MAX_VIEWS];
    int nviews;
    int total_items;
    int rb;                // rows per band (even)
    float w0, w1, w2;      // blur taps: centre, +-1, +-2
    float *E;
    uint8_t *mask;
    float *median_out;
    unsigned *hist1;       // [V][kBins1]
    unsigned *hist2;       // [V][kBins2] bits [18:9] of the candidates
    unsigned *sel;         // [V][4]: kept count, median bin of bits [30:19], count below that bin
    unsigned *cand_count;  // [V]
    float *cand;           // candidate values, laid out like E
    unsigned *med_bits;    // [V]: bits of the median of M^2
    float *kept;           // [item][kItemCols * rb]: kept M^2, row pair after row pair (lane, row, column)
    uint8_t *kmask;        // [item][rb / 2][32]: keep bits of each lane's 4 columns x 2 rows
    unsigned *kcount;      // [item]: kept values of the item
    unsigned *bar;         // grid barrier state [2]
    int32_t *status;
    long long spin_limit;  // grid-barrier polls
    int expire;            // test hook: bit 0 withholds the first grid barrier
};

// Shared memory of a walk block, one layout per phase.
union alignas(16) WalkSmem {
    unsigned hist[kWWarps][kBins1 / 2];  // A: warp histograms of bits [30:19], two 16-bit counts a word
    struct {
        unsigned h2[kWWarps][kBins2];    // B: warp counts of bits [18:9] of the candidates
        float cbuf[kWWarps][kBCand];     //    candidates waiting for their reservation
    } b;
    unsigned hist3[kBins3];              // C: count of bits [8:0]
    struct {
        float vals[kWWarps][2 * kDPairs * 2 * kItemCols];  // D: E of two chunks' kept values
        float row[kWWarps][2][32 * kQ];                //    E rows of a pair, for coalesced stores
        uint8_t mrow[kWWarps][2][32 * kQ];             //    NMS mask rows of a pair
    } d;
};

// 4-byte asynchronous copies into shared memory (phase D stages a chunk's kept
// values with every copy in flight at once, one commit group per chunk).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// waits until at most N of this thread's commit groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void item_origin(const EdgeArgs &a, int it, int &v, int &xg, int &y0)
{
    v = 0;
    while (v + 1 < a.nviews && a.v[v + 1].item_base <= it) ++v;
    const EdgeView &V = a.v[v];
    const int li = it - V.item_base;
    const int band = li / V.groups;
    xg = (li - band * V.groups) * kItemCols;
    y0 = band * a.rb;
}

// Per-lane constants of an item's walk.
struct QLane {
    const uint8_t *rgb;
    long long pitch;
    int w, h;
    int cx;             // first of the lane's 4 columns (may lie outside the image)
    int y0, nout, nin;  // first output row, output rows, input rows (nout + 8)
    unsigned bits;      // bits 0-3: columns inside the image; 4-7: columns this lane outputs
                        // (lanes 1..30, inside the image); 8: all 4 inside (word loads)
};

// The raw words of the lane's 4 pixels of input row i (image row y0 - 4 + i,
// clamped).  Fast lanes: the aligned words covering their 12 bytes and the
// byte shift of the first; other lanes: one word per pixel (clamped column).
__device__ __forceinline__ void load_row(const QLane &q, int i, unsigned (&w)[4], unsigned &shift)
{
    const int y = clampi(q.y0 - 4 + i, 0, q.h - 1);
    const uint8_t *row = q.rgb + (long long)y * q.pitch;
    if (q.bits & 0x100u) {
        const uintptr_t p = reinterpret_cast<uintptr_t>(row + 3 * q.cx);
        const unsigned *wp = reinterpret_cast<const unsigned *>(p & ~uintptr_t(3));
        shift = unsigned(p & 3) * 8u;
        w[0] = __ldg(wp);
        w[1] = __ldg(wp + 1);
        w[2] = __ldg(wp + 2);
        // the fourth word holds the last byte only when the span is not word aligned
        w[3] = shift ? __ldg(wp + 3) : 0u;
    } else {
        shift = 0u;
#pragma unroll
        for (int j = 0; j < kQ; ++j) {
            const uint8_t *b = row + 3 * clampi(q.cx + j, 0, q.w - 1);
            w[j] = unsigned(b[0]) | unsigned(b[1]) << 8 | unsigned(b[2]) << 16;
        }
    }
}

__device__ __forceinline__ void row_luma(const QLane &q, const unsigned (&w)[4], unsigned shift, float (&I)[kQ])
{
    unsigned px[kQ];
    if (q.bits & 0x100u) {
        const unsigned u0 = __funnelshift_r(w[0], w[1], shift);
        const unsigned u1 = __funnelshift_r(w[1], w[2], shift);
        const unsigned u2 = __funnelshift_r(w[2], w[3], shift);
        px[0] = u0;
        px[1] = __byte_perm(u0, u1, 0x6543);
        px[2] = __byte_perm(u1, u2, 0x5432);
        px[3] = u2 >> 8;
    } else {
#pragma unroll
        for (int j = 0; j < kQ; ++j) px[j] = w[j];
    }
#pragma unroll
    for (int j = 0; j < kQ; ++j) I[j] = luma_exact(px[j]);
}

// Walk state of a lane.
struct QState {
    float I0[kQ], I1[kQ];      // luma of input rows i - 2, i - 1
    float2 acc[4][kQ];         // vertical blur chains: acc[d] lacks the d + 1 newest blurred rows
    float M0[kQ + 2];          // M^2 of NMS row q - 1 (index 0: column -1, kQ + 1: column kQ)
    float M1[kQ + 2];          // M^2 of NMS row q
    unsigned dir1;             // direction class of row q: 4 bits per column (see dir_bits)
    unsigned w[4], shift;      // words of the next input row
    unsigned keep0;            // keep bits of the first row of a pair, waiting for the second
};

// Direction class of a blurred gradient for NMS, 4 bits: horizontal (|gy| <=
// tan 22.5 |gx|), vertical (|gx| <= tan 22.5 |gy|; read only when not
// horizontal), same signs (gx > 0 == gy > 0), and whether the + direction
// neighbour (compared with >=) is the right one (horizontal: gx > 0) or the
// one in the row below (otherwise: gy > 0).
__device__ __forceinline__ unsigned dir_bits(float2 g)
{
    const float ax = fabsf(g.x), ay = fabsf(g.y);
    const bool gxp = g.x > 0.f, gyp = g.y > 0.f;
    const bool horiz = ay <= __fmul_rn(kTan22, ax);
    const bool vert = ax <= __fmul_rn(kTan22, ay);
    const bool same = gxp == gyp;
    const bool pos = horiz ? gxp : gyp;
    return unsigned(horiz) | unsigned(vert) << 1 | unsigned(same) << 2 | unsigned(pos) << 3;
}

// Output of phase A for one item.
struct QOut {
    float *slot;       // the item's kept values
    uint8_t *km;       // the item's keep masks
    unsigned *whist;   // the warp's histogram
    unsigned run;      // kept values so far
    unsigned cap;      // kItemCols * rb
    int32_t *status;
};

__device__ __forceinline__ void emit_pair(QOut &o, int pair, unsigned k8, const float (&vv)[2 * kQ])
{
    const int lane = threadIdx.x & 31;
    unsigned excl;
    const unsigned tot = warp_exclusive_scan(__popc(k8), &excl);
    unsigned at = o.run + excl;
#pragma unroll
    for (int b = 0; b < 2 * kQ; ++b) {
        const bool kb = (k8 >> b & 1u) != 0u;
        if (kb) {
            if (GSP_BOUND(at, o.cap, o.status)) o.slot[at] = vv[b];
            const unsigned bin = __float_as_uint(vv[b]) >> kShift1;
            atomicAdd(&o.whist[bin >> 1], 1u << ((bin & 1u) << 4));
        }
        at += kb;
    }
    o.km[pair * 32 + lane] = uint8_t(k8);
    o.run += tot;
}

// Input step i of the walk (PAR = i mod 2): luma row i, Sobel row i - 1 and its
// horizontal blur, which completes the vertical blur of row m = y0 - 7 + i
// (i >= 6) and its M^2, then (i >= 8) NMS of output row r = i - 8, emitted
// with the row before it when r is odd.  The vertical blur of a row is the
// chain w2 h0 (+) w1 h1 (+) w0 h2 (+) w1 h3 (+) w2 h4 over its five blurred
// rows, oldest first: four partial chains advance in place as rows arrive.
template <int PAR>
__device__ __forceinline__ void qstep(const QLane &q, const float2 w0v, const float2 w1v, const float2 w2v,
                                      QState &s, QOut &o, int i)
{
    float Ic[kQ];
    row_luma(q, s.w, s.shift, Ic);
    if (i + 1 < q.nin) load_row(q, i + 1, s.w, s.shift);
    float2 g[kQ];
    if (i >= 2) {
        // vertical parts of Sobel row i - 1 (exact integers in FP32), the lane's
        // columns at index 1..4, the neighbours' edge columns at 0 and 5
        float v121[kQ + 2], vd[kQ + 2];
#pragma unroll
        for (int j = 0; j < kQ; ++j) {
            v121[j + 1] = __fadd_rn(__fmaf_rn(2.f, s.I1[j], s.I0[j]), Ic[j]);
            vd[j + 1] = __fsub_rn(Ic[j], s.I0[j]);
        }
        v121[0] = __shfl_up_sync(kFull, v121[kQ], 1);
        vd[0] = __shfl_up_sync(kFull, vd[kQ], 1);
        v121[kQ + 1] = __shfl_down_sync(kFull, v121[1], 1);
        vd[kQ + 1] = __shfl_down_sync(kFull, vd[1], 1);
        // (Sx, Sy) at columns -2 .. kQ + 1 (index + 2)
        float2 f[kQ + 4];
#pragma unroll
        for (int j = 0; j < kQ; ++j)
            f[j + 2] = make_float2(__fsub_rn(v121[j + 2], v121[j]),
                                   __fadd_rn(__fmaf_rn(2.f, vd[j + 1], vd[j]), vd[j + 2]));
        f[0].x = __shfl_up_sync(kFull, f[kQ].x, 1);
        f[0].y = __shfl_up_sync(kFull, f[kQ].y, 1);
        f[1].x = __shfl_up_sync(kFull, f[kQ + 1].x, 1);
        f[1].y = __shfl_up_sync(kFull, f[kQ + 1].y, 1);
        f[kQ + 2].x = __shfl_down_sync(kFull, f[2].x, 1);
        f[kQ + 2].y = __shfl_down_sync(kFull, f[2].y, 1);
        f[kQ + 3].x = __shfl_down_sync(kFull, f[3].x, 1);
        f[kQ + 3].y = __shfl_down_sync(kFull, f[3].y, 1);
#pragma unroll
        for (int j = 0; j < kQ; ++j) {
            // horizontal blur, taps paired (both components at once)
            const float2 h = __ffma2_rn(w2v, __fadd2_rn(f[j], f[j + 4]),
                                        __ffma2_rn(w1v, __fadd2_rn(f[j + 1], f[j + 3]), __fmul2_rn(w0v, f[j + 2])));
            // the newest row ends the oldest chain and enters the others
            g[j] = __ffma2_rn(w2v, h, s.acc[3][j]);
            s.acc[3][j] = __ffma2_rn(w1v, h, s.acc[2][j]);
            s.acc[2][j] = __ffma2_rn(w0v, h, s.acc[1][j]);
            s.acc[1][j] = __ffma2_rn(w1v, h, s.acc[0][j]);
            s.acc[0][j] = __fmul2_rn(w2v, h);
        }
    }
#pragma unroll
    for (int j = 0; j < kQ; ++j) {
        s.I0[j] = s.I1[j];
        s.I1[j] = Ic[j];
    }
    if (i < 6) return;
    const int m = q.y0 - 7 + i;
    const bool row_in = m >= 0 && m < q.h;
    float M2[kQ + 2];
#pragma unroll
    for (int j = 0; j < kQ; ++j)
        M2[j + 1] = (row_in && (q.bits >> j & 1u)) ? __fmaf_rn(g[j].x, g[j].x, __fmul_rn(g[j].y, g[j].y)) : 0.f;
    M2[0] = __shfl_up_sync(kFull, M2[kQ], 1);
    M2[kQ + 1] = __shfl_down_sync(kFull, M2[1], 1);
    if (i >= 8) {
        // NMS of row q (M0 = q - 1, M1 = q, M2 = q + 1); column j is index j + 1.
        // The neighbour in the + direction of the gradient (compared with >=)
        // and the one in the - direction (compared with >): along the row for
        // the horizontal class (+ is +x when gx > 0); otherwise in row q + 1
        // exactly when gy > 0, at the column offset of the class.
        unsigned keep = 0u;
#pragma unroll
        for (int j = 0; j < kQ; ++j) {
            const int k = j + 1;
            const unsigned d = s.dir1 >> (4 * j);
            const bool horiz = d & 1u, vert = d & 2u, same = d & 4u, pos = d & 8u;
            const float mq = s.M1[k];
            const float n0 = vert ? s.M0[k] : (same ? s.M0[k - 1] : s.M0[k + 1]);
            const float n2 = vert ? M2[k] : (same ? M2[k + 1] : M2[k - 1]);
            const float lo = horiz ? s.M1[k - 1] : n0, hi = horiz ? s.M1[k + 1] : n2;
            const float mp = pos ? hi : lo, mm = pos ? lo : hi;
            keep |= unsigned(mq > 0.f && mq >= mp && mq > mm) << j;
        }
        keep &= (q.bits >> 4) & 0xfu;
        const int r = i - 8;
        if (PAR == 0 && r + 1 < q.nout) {
            s.keep0 = keep;
        } else {
            // the pair's values: the first row's M^2 is row q - 1 (M0) on the
            // second step of the pair, the second row's is row q (M1)
            float vv[2 * kQ];
            unsigned k8;
            if (PAR == 1) {
                k8 = s.keep0 | keep << kQ;
#pragma unroll
                for (int j = 0; j < kQ; ++j) {
                    vv[j] = s.M0[j + 1];
                    vv[kQ + j] = s.M1[j + 1];
                }
            } else {
                k8 = keep;
#pragma unroll
                for (int j = 0; j < kQ; ++j) {
                    vv[j] = s.M1[j + 1];
                    vv[kQ + j] = 0.f;
                }
            }
            emit_pair(o, r >> 1, k8, vv);
        }
    }
#pragma unroll
    for (int k = 0; k < kQ + 2; ++k) {
        s.M0[k] = s.M1[k];
        s.M1[k] = M2[k];
    }
    unsigned dir = 0u;
#pragma unroll
    for (int j = 0; j < kQ; ++j) dir |= dir_bits(g[j]) << (4 * j);
    s.dir1 = dir;
}

// Phase A of one warp item: walk the band, compact the kept values per row
// pair, count them in the warp histogram.  Returns the item's kept count.
__device__ unsigned walk_item(const EdgeArgs &a, int it, unsigned *whist)
{
    int v, xg, y0;
    item_origin(a, it, v, xg, y0);
    const EdgeView &V = a.v[v];
    const int lane = threadIdx.x & 31;
    QLane q;
    q.rgb = V.rgb;
    q.pitch = V.pitch;
    q.w = V.w;
    q.h = V.h;
    q.cx = xg - kQ + kQ * lane;
    q.y0 = y0;
    q.nout = min(a.rb, V.h - y0);
    q.nin = q.nout + 8;
    unsigned colmask = 0u;
#pragma unroll
    for (int j = 0; j < kQ; ++j) colmask |= unsigned(q.cx + j >= 0 && q.cx + j < V.w) << j;
    q.bits = colmask | ((lane >= 1 && lane <= 30) ? colmask : 0u) << 4 |
             unsigned(q.cx >= 0 && q.cx + kQ <= V.w) << 8;
    QOut o;
    o.slot = a.kept + (size_t)it * kItemCols * a.rb;
    o.km = a.kmask + (size_t)it * (a.rb / 2) * 32;
    o.whist = whist;
    o.run = 0;
    o.cap = unsigned(kItemCols * a.rb);
    o.status = a.status;
    const float2 w0v = make_float2(a.w0, a.w0), w1v = make_float2(a.w1, a.w1), w2v = make_float2(a.w2, a.w2);
    QState s;
    s.keep0 = 0u;
    load_row(q, 0, s.w, s.shift);
#pragma unroll 1
    for (int i = 0; i < q.nin; i += 2) {
        qstep<0>(q, w0v, w1v, w2v, s, o, i);
        if (i + 1 < q.nin) qstep<1>(q, w0v, w1v, w2v, s, o, i + 1);
    }
    if (lane == 0) a.kcount[it] = o.run;
    return o.run;
}

// Add a warp histogram (two 16-bit counts a word) to view v's global
// histogram and clear it.
__device__ __forceinline__ void flush_whist(unsigned *whist, unsigned *gh)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int b = lane; b < kBins1 / 2; b += 32) {
        const unsigned c = whist[b];
        if (c) {
            if (c & 0xffffu) atomicAdd(gh + 2 * b, c & 0xffffu);
            if (c >> 16) atomicAdd(gh + 2 * b + 1, c >> 16);
            whist[b] = 0u;
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(WNT, kWalkBlocksPerSM) edge_walk_kernel(const __grid_constant__ EdgeArgs a)
{
    __shared__ WalkSmem sm;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x;
    const long long gw = (long long)blockIdx.x * kWWarps + wid, nw = (long long)G * kWWarps;
    const int it_begin = int(a.total_items * gw / nw), it_end = int(a.total_items * (gw + 1) / nw);

    // ---- phase A: stencil walk, NMS, compacted kept M^2, warp histograms of bits [30:19]
    {
        unsigned *whist = sm.hist[wid];
        for (int b = lane; b < kBins1 / 2; b += 32) whist[b] = 0u;
        __syncwarp();
        int cur_view = -1;
        unsigned since = 0;  // kept values counted since the last flush (16-bit counts)
        const unsigned item_cap = unsigned(kItemCols * a.rb);
        for (int it = it_begin; it < it_end; ++it) {
            int v = 0;
            while (v + 1 < a.nviews && a.v[v + 1].item_base <= it) ++v;
            if (v != cur_view || since + item_cap > 0xffffu) {
                if (cur_view >= 0) flush_whist(whist, a.hist1 + (size_t)cur_view * kBins1);
                cur_view = v;
                since = 0;
            }
            since += walk_item(a, it, whist);
        }
        if (cur_view >= 0) flush_whist(whist, a.hist1 + (size_t)cur_view * kBins1);
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status, (a.expire & 1) != 0)) return;

    // ---- phase B0: each view's median bin of bits [30:19] and kept count (block v)
    // (thread t holds bins [32 t, 32 t + 32) in registers: eight 16-byte loads,
    // one block scan, and the thread whose range holds the median rank walks it)
    for (int v = blockIdx.x; v < a.nviews; v += G) {
        static_assert(kBins1 == 32 * WNT, "32 bins per thread");
        const uint4 *h4 = reinterpret_cast<const uint4 *>(a.hist1 + (size_t)v * kBins1) + tid * 8;
        unsigned hb[32];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint4 u = __ldcg(h4 + k);
            hb[4 * k] = u.x; hb[4 * k + 1] = u.y; hb[4 * k + 2] = u.z; hb[4 * k + 3] = u.w;
        }
        unsigned seg = 0;
#pragma unroll
        for (int k = 0; k < 32; ++k) seg += hb[k];
        unsigned before;
        const unsigned n = block_exclusive_scan<WNT>(seg, &before);
        const unsigned rank = n > 0 ? (n - 1) / 2 : 0u;
        if (tid == 0) a.sel[4 * v + 0] = n;
        if (n > 0 && rank >= before && rank < before + seg) {
            unsigned acc = before;
            int b1 = 0;
            unsigned below = 0;
            bool found = false;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                if (!found && rank < acc + hb[k]) {
                    b1 = 32 * tid + k;
                    below = acc;
                    found = true;
                }
                acc += hb[k];
            }
            a.sel[4 * v + 1] = unsigned(b1);
            a.sel[4 * v + 2] = below;
        }
        if (n == 0 && tid == 0) {
            a.sel[4 * v + 1] = 0u;
            a.sel[4 * v + 2] = 0u;
        }
        __syncthreads();
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status)) return;

    // ---- phase B: each warp streams its items' kept values, collects the
    // candidates (values in the median bin) with their count on bits [18:9],
    // and appends them to the view's list with one reservation per buffer
    {
        unsigned *h2s = sm.b.h2[wid];
        float *cbuf = sm.b.cbuf[wid];
        for (int b = lane; b < kBins2; b += 32) h2s[b] = 0u;
        __syncwarp();
        int cur_view = -1;
        for (int it = it_begin; it < it_end; ++it) {
            int v = 0;
            while (v + 1 < a.nviews && a.v[v + 1].item_base <= it) ++v;
            if (v != cur_view) {
                if (cur_view >= 0) {
                    unsigned *h2 = a.hist2 + (size_t)cur_view * kBins2;
                    for (int b = lane; b < kBins2; b += 32) {
                        const unsigned c = h2s[b];
                        if (c) {
                            atomicAdd(h2 + b, c);
                            h2s[b] = 0u;
                        }
                    }
                    __syncwarp();
                }
                cur_view = v;
            }
            const unsigned b1 = __ldcg(a.sel + 4 * v + 1);
            const unsigned n = __ldcg(a.kcount + it);
            const float *src = a.kept + (size_t)it * kItemCols * a.rb;
            float *cand = a.cand + a.v[v].out_off;
            [[maybe_unused]] const long long vpx = (long long)a.v[v].w * a.v[v].h;
            unsigned nc = 0;  // candidates buffered
            constexpr int kBLoads = 16;  // values per lane in flight
            for (unsigned c0 = 0; c0 < n; c0 += kBLoads * 32) {
                float val[kBLoads];
#pragma unroll
                for (int k = 0; k < kBLoads; ++k) {
                    const unsigned e = c0 + 32 * k + lane;
                    val[k] = e < n ? __ldcg(src + e) : 0.f;
                }
#pragma unroll
                for (int k = 0; k < kBLoads; ++k) {
                    const unsigned e = c0 + 32 * k + lane;
                    const unsigned bits = __float_as_uint(val[k]);
                    const bool pick = e < n && (bits >> kShift1) == b1;
                    const unsigned m = __ballot_sync(kFull, pick);
                    if (!m) continue;
                    if (nc + 32 > unsigned(kBCand)) {
                        unsigned at = 0;
                        if (lane == 0) at = atomicAdd(a.cand_count + v, nc);
                        at = __shfl_sync(kFull, at, 0);
                        __syncwarp();
                        for (unsigned j = lane; j < nc; j += 32)
                            if (GSP_BOUND(at + j, vpx, a.status)) cand[at + j] = cbuf[j];
                        nc = 0;
                        __syncwarp();
                    }
                    if (pick) {
                        cbuf[nc + __popc(m & ((1u << lane) - 1u))] = val[k];
                        atomicAdd(&h2s[(bits >> kShift2) & (kBins2 - 1)], 1u);
                    }
                    nc += __popc(m);
                }
            }
            __syncwarp();
            if (nc) {
                unsigned at = 0;
                if (lane == 0) at = atomicAdd(a.cand_count + v, nc);
                at = __shfl_sync(kFull, at, 0);
                for (unsigned j = lane; j < nc; j += 32)
                    if (GSP_BOUND(at + j, vpx, a.status)) cand[at + j] = cbuf[j];
                __syncwarp();
            }
        }
        if (cur_view >= 0) {
            unsigned *h2 = a.hist2 + (size_t)cur_view * kBins2;
            for (int b = lane; b < kBins2; b += 32) {
                const unsigned c = h2s[b];
                if (c) atomicAdd(h2 + b, c);
            }
        }
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status)) return;

    // ---- phase C: exact median of each view (block v): the level-2 bin from
    // the candidates' count, then bits [8:0] among the candidates in it
    for (int v = blockIdx.x; v < a.nviews; v += G) {
        const unsigned n = a.sel[4 * v + 0];
        unsigned bits = 0;
        if (n > 0) {
            const unsigned b1 = a.sel[4 * v + 1];
            unsigned rank = (n - 1) / 2 - a.sel[4 * v + 2];
            int b2;
            unsigned below2;
            block_find_bin<WNT>(a.hist2 + (size_t)v * kBins2, kBins2, rank, &b2, &below2);
            rank -= below2;
            for (int i = tid; i < kBins3; i += WNT) sm.hist3[i] = 0;
            __syncthreads();
            const float *cand = a.cand + a.v[v].out_off;
            const unsigned count = a.cand_count[v];
            constexpr int kCLoads = 8;  // candidates per thread in flight
            for (unsigned i0 = 0; i0 < count; i0 += kCLoads * WNT) {
                unsigned cb[kCLoads];
#pragma unroll
                for (int u = 0; u < kCLoads; ++u) {
                    const unsigned i = i0 + u * WNT + tid;
                    cb[u] = i < count ? __float_as_uint(__ldcg(cand + i)) : 0xffffffffu;
                }
#pragma unroll
                for (int u = 0; u < kCLoads; ++u)
                    if (cb[u] != 0xffffffffu && ((cb[u] >> kShift2) & (kBins2 - 1)) == unsigned(b2))
                        atomicAdd(&sm.hist3[cb[u] & (kBins3 - 1)], 1u);
            }
            __syncthreads();
            int b3;
            unsigned below3;
            block_find_bin<WNT>(sm.hist3, kBins3, rank, &b3, &below3);
            bits = (b1 << kShift1) | (unsigned(b2) << kShift2) | unsigned(b3);
        }
        if (tid == 0) {
            a.med_bits[v] = bits;
            a.median_out[v] = __fsqrt_rn(__uint_as_float(bits)) * (1.0f / 255000.0f);
        }
        __syncthreads();
    }
    if (!grid_barrier(a.bar, G, a.spin_limit, a.status)) return;

    // ---- phase D: every warp writes its items' E rows, zeros and sqrt(M^2) /
    // median.  Row pairs go in chunks of kDPairs, pipelined: while chunk c is
    // written, the kept values of chunk c + 1 are on their way into the other
    // shared buffer (cp.async) and the keep bytes of chunk c + 2 are loading.
    // A chunk's kept values are converted to E by all lanes together (no lane
    // idles on a pixel it does not keep), then each row is staged in shared
    // memory so that every store instruction covers contiguous columns.
    {
        float *vbuf = sm.d.vals[wid];  // two buffers of kDPairs * 2 * kItemCols values
        constexpr int kDBuf = kDPairs * 2 * kItemCols;
        for (int it = it_begin; it < it_end; ++it) {
            int v, xg, y0;
            item_origin(a, it, v, xg, y0);
            const EdgeView &V = a.v[v];
            const float med2 = __uint_as_float(__ldcg(a.med_bits + v));
            const float smed = __fsqrt_rn(med2);
            const int nout = min(a.rb, V.h - y0);
            const int npairs = (nout + 1) / 2;
            const int nch = (npairs + kDPairs - 1) / kDPairs;
            const float *src = a.kept + (size_t)it * kItemCols * a.rb;
            const uint8_t *km = a.kmask + (size_t)it * (a.rb / 2) * 32;
            auto load_masks = [&](int c, unsigned (&k8)[kDPairs]) {
#pragma unroll
                for (int r = 0; r < kDPairs; ++r) {
                    const int t = c * kDPairs + r;
                    k8[r] = t < npairs ? unsigned(__ldcg(km + t * 32 + lane)) : 0u;
                }
            };
            auto scan = [&](const unsigned (&k8)[kDPairs], unsigned (&excl)[kDPairs], unsigned (&off)[kDPairs]) {
                unsigned tot = 0;
#pragma unroll
                for (int r = 0; r < kDPairs; ++r) {
                    off[r] = tot;
                    tot += warp_exclusive_scan(__popc(k8[r]), &excl[r]);
                }
                return tot;
            };
            auto issue = [&](float *dst, unsigned from, unsigned n) {
                __syncwarp();
                for (unsigned j = lane; j < n; j += 32) cp_async4(dst + j, src + from + j);
                cp_async_commit();
            };
            unsigned ck8[kDPairs], cex[kDPairs], cof[kDPairs], nk8[kDPairs];
            load_masks(0, ck8);
            unsigned ctot = scan(ck8, cex, cof);
            unsigned run = 0;
            issue(vbuf, 0, ctot);
            if (nch > 1) load_masks(1, nk8);
            for (int c = 0; c < nch; ++c) {
                float *cur = vbuf + (c & 1) * kDBuf;
                unsigned xex[kDPairs], xof[kDPairs], xtot = 0;
                if (c + 1 < nch) {
                    xtot = scan(nk8, xex, xof);
                    issue(vbuf + ((c + 1) & 1) * kDBuf, run + ctot, xtot);
                    cp_async_wait<1>();  // chunk c has landed, chunk c + 1 may still fly
                } else {
                    cp_async_wait<0>();
                }
                unsigned xk8[kDPairs];
#pragma unroll
                for (int r = 0; r < kDPairs; ++r) xk8[r] = nk8[r];
                if (c + 2 < nch) load_masks(c + 2, nk8);
                __syncwarp();
                for (unsigned j = lane; j < ctot; j += 32)
                    cur[j] = med2 > 0.f ? __fdiv_rn(__fsqrt_rn(cur[j]), smed) : 0.f;
                __syncwarp();
#pragma unroll
                for (int r = 0; r < kDPairs; ++r) {
                    const int t = c * kDPairs + r;
                    if (t >= npairs) break;
                    const float *p = cur + cof[r] + cex[r];
                    float e[2 * kQ];
#pragma unroll
                    for (int b = 0; b < 2 * kQ; ++b) {
                        e[b] = 0.f;
                        if (ck8[r] >> b & 1u) e[b] = *p++;
                    }
                    float *row0 = sm.d.row[wid][0], *row1 = sm.d.row[wid][1];
                    reinterpret_cast<float4 *>(row0)[lane] = make_float4(e[0], e[1], e[2], e[3]);
                    reinterpret_cast<float4 *>(row1)[lane] = make_float4(e[4], e[5], e[6], e[7]);
                    if (a.mask) {
                        unsigned lo = 0, hi = 0;
#pragma unroll
                        for (int j = 0; j < kQ; ++j) {
                            lo |= (ck8[r] >> j & 1u) << (8 * j);
                            hi |= (ck8[r] >> (j + kQ) & 1u) << (8 * j);
                        }
                        reinterpret_cast<unsigned *>(sm.d.mrow[wid][0])[lane] = lo;
                        reinterpret_cast<unsigned *>(sm.d.mrow[wid][1])[lane] = hi;
                    }
                    __syncwarp();
                    for (int rr = 0; rr < 2; ++rr) {
                        const int qrow = 2 * t + rr;
                        if (qrow >= nout) break;
                        const long long rowoff = V.out_off + (long long)(y0 + qrow) * V.w + xg;
                        float *out = a.E + rowoff;
                        uint8_t *mout = a.mask ? a.mask + rowoff : nullptr;
                        const float *st = sm.d.row[wid][rr];
                        const uint8_t *mst = sm.d.mrow[wid][rr];
#pragma unroll
                        for (int k = 0; k < kQ; ++k) {
                            const int cc = 32 * k + lane - kQ;  // output column xg + cc, staged at cc + kQ
                            if (cc >= 0 && cc < kItemCols && xg + cc < V.w) {
                                out[cc] = st[cc + kQ];
                                if (mout) mout[cc] = mst[cc + kQ];
                            }
                        }
                    }
                    __syncwarp();
                }
                run += ctot;
                ctot = xtot;
#pragma unroll
                for (int r = 0; r < kDPairs; ++r) {
                    ck8[r] = xk8[r];
                    cex[r] = xex[r];
                    cof[r] = xof[r];
                }
            }
        }
    }
}

// ------------------------------------------------------------ plain path

struct PlainBufs {
    int *I;          // (h+8) x (w+8)
    float *Sx, *Sy;  // (h+6) x (w+6)
    float *Hx, *Hy;  // (h+6) x (w+2)
    float *Gx, *Gy, *M;  // (h+2) x (w+2)
    unsigned *hist;  // kBins1
    unsigned *state; // [0] prefix bits, [1] remaining rank, [2] count
};

__global__ void plain_luma(TileView V, int *I)
{
    int W = V.w + 8, H = V.h + 8;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    int r = int(i / W), c = int(i - (long long)r * W);
    int yy = clampi(r - 4, 0, V.h - 1), xx = clampi(c - 4, 0, V.w - 1);
    const uint8_t *p = V.rgb + (long long)yy * V.pitch + 3 * xx;
    I[i] = 299 * int(p[0]) + 587 * int(p[1]) + 114 * int(p[2]);
}

__global__ void plain_sobel(TileView V, const int *I, float *Sx, float *Sy)
{
    int W = V.w + 6, H = V.h + 6, IWp = V.w + 8;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    int r = int(i / W), c = int(i - (long long)r * W);
    const int *a0 = I + (long long)r * IWp + c, *a1 = a0 + IWp, *a2 = a1 + IWp;
    int sx = (a0[2] - a0[0]) + 2 * (a1[2] - a1[0]) + (a2[2] - a2[0]);
    int sy = (a2[0] - a0[0]) + 2 * (a2[1] - a0[1]) + (a2[2] - a0[2]);
    Sx[i] = float(sx);
    Sy[i] = float(sy);
}

__global__ void plain_hblur(TileView V, const float *Sx, const float *Sy, float *Hx, float *Hy, float w0,
                            float w1, float w2)
{
    int W = V.w + 2, H = V.h + 6, SWp = V.w + 6;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    int r = int(i / W), c = int(i - (long long)r * W);
    const float *x = Sx + (long long)r * SWp + c, *y = Sy + (long long)r * SWp + c;
    Hx[i] = __fmaf_rn(w2, x[0] + x[4], __fmaf_rn(w1, x[1] + x[3], __fmul_rn(w0, x[2])));
    Hy[i] = __fmaf_rn(w2, y[0] + y[4], __fmaf_rn(w1, y[1] + y[3], __fmul_rn(w0, y[2])));
}

__global__ void plain_vblur_mag(TileView V, const float *Hx, const float *Hy, float *Gx, float *Gy,
                                float *M, float w0, float w1, float w2)
{
    int W = V.w + 2, H = V.h + 2;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)W * H) return;
    int r = int(i / W), c = int(i - (long long)r * W);
    long long s = (long long)W;
    const float *x = Hx + (long long)r * W + c, *y = Hy + (long long)r * W + c;
    float gx = vblur5(x[0], x[s], x[2 * s], x[3 * s], x[4 * s], w0, w1, w2);
    float gy = vblur5(y[0], y[s], y[2 * s], y[3 * s], y[4 * s], w0, w1, w2);
    bool inside = r >= 1 && r <= V.h && c >= 1 && c <= V.w;
    Gx[i] = gx;
    Gy[i] = gy;
    M[i] = inside ? __fmaf_rn(gx, gx, __fmul_rn(gy, gy)) : 0.f;  // squared magnitude
}

__global__ void plain_nms(TileView V, const float *Gx, const float *Gy, const float *M, float *E,
                          uint8_t *mask)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)V.w * V.h) return;
    int y = int(i / V.w), x = int(i - (long long)y * V.w);
    int W = V.w + 2;
    long long q = (long long)(y + 1) * W + (x + 1);
    float m = M[q], gx = Gx[q], gy = Gy[q];
    float ax = fabsf(gx), ay = fabsf(gy);
    bool horiz = ay <= __fmul_rn(kTan22, ax);
    bool vert = !horiz && ax <= __fmul_rn(kTan22, ay);
    int sx = vert ? 0 : (gx > 0.f) - (gx < 0.f);
    int sy = horiz ? 0 : (gy > 0.f) - (gy < 0.f);
    float mp = M[q + (long long)sy * W + sx], mm = M[q - (long long)sy * W - sx];
    bool keep = m > 0.f && m >= mp && m > mm;
    E[V.out_off + i] = keep ? m : 0.f;
    if (mask) mask[V.out_off + i] = keep;
}

// Histogram of digit (bits >> shift) & (nbins-1) over kept values whose bits
// above the digit match state[0] (pass > 0).
__global__ void plain_hist(const float *E, long long n, int shift, int nbins, int pass,
                           const unsigned *state, unsigned *hist)
{
    __shared__ unsigned h[kBins1];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    unsigned prefix = pass ? state[0] : 0;
    int hi = shift + __popc(nbins - 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v = E[i];
        if (!(v > 0.f)) continue;
        unsigned b = __float_as_uint(v);
        if (pass && (b >> hi) != (prefix >> hi)) continue;
        atomicAdd(&h[(b >> shift) & (nbins - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void __launch_bounds__(NT) plain_select(unsigned *hist, int nbins, int shift, int pass,
                                                   unsigned *state, unsigned *med_bits, float *median_out)
{
    unsigned seg = 0;
    const int per = nbins / NT;
    for (int k = 0; k < per; ++k) seg += hist[threadIdx.x * per + k];
    unsigned before;
    unsigned n = block_exclusive_scan(seg, &before);
    if (pass == 0) {
        if (threadIdx.x == 0) {
            state[2] = n;
            state[1] = n ? (n - 1) / 2 : 0;
            state[0] = 0;
        }
        __syncthreads();
    }
    if (state[2] == 0) {
        if (threadIdx.x == 0 && pass == 2) {
            *med_bits = 0;
            *median_out = 0.f;
        }
        return;
    }
    int bin;
    unsigned below;
    block_find_bin(hist, nbins, state[1], &bin, &below);
    if (threadIdx.x == 0) {
        state[0] |= unsigned(bin) << shift;
        state[1] -= below;
        if (pass == 2) {
            *med_bits = state[0];
            *median_out = __fsqrt_rn(__uint_as_float(state[0])) * (1.0f / 255000.0f);
        }
    }
}

__global__ void plain_normalise(TileView V, float *E, const unsigned *med_bits)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)V.w * V.h) return;
    const float med2 = __uint_as_float(*med_bits);
    const float m2 = E[V.out_off + i];
    if (med2 > 0.f && m2 > 0.f) E[V.out_off + i] = __fdiv_rn(__fsqrt_rn(m2), __fsqrt_rn(med2));
}

void fill_taps(const gsp_edge_opts &o, float &w0, float &w1, float &w2)
{
    if (o.use_custom_taps) {
        w0 = o.taps[2];
        w1 = o.taps[1];
        w2 = o.taps[0];
        return;
    }
    double s = o.sigma > 0 ? o.sigma : 1.0;
    double e1 = exp(-1.0 / (2 * s * s)), e2 = exp(-4.0 / (2 * s * s));
    double z = 1.0 + 2 * e1 + 2 * e2;
    w0 = float(1.0 / z);
    w1 = float(e1 / z);
    w2 = float(e2 / z);
}

// Work plan of the walk kernel: kWalkBlocksPerSM blocks of WNT threads per SM;
// warp items of 120 output columns x rb rows (rb even).  rb minimises the
// rounds of items over the warps times the rows a round walks (each band
// re-walks 8 halo rows).
struct EdgePlan {
    int rb = 0;
    long long items = 0;
};

long long plan_items(const gsp_image_desc *imgs, int nv, int rb)
{
    long long n = 0;
    for (int v = 0; v < nv; ++v)
        n += (long long)div_up(imgs[v].width, kItemCols) * (long long)div_up(imgs[v].height, rb);
    return n;
}

EdgePlan edge_plan(const gsp_image_desc *imgs, int nv)
{
    EdgePlan p;
    const long long warps = (long long)num_sms() * kWalkBlocksPerSM * kWWarps;
    double best = 1e300;
    for (int rb = 8; rb <= 128; rb += 2) {
        const long long items = plan_items(imgs, nv, rb);
        const double cost = double((items + warps - 1) / warps) * double(rb + 8);
        if (cost < best) {
            best = cost;
            p.rb = rb;
            p.items = items;
        }
    }
    return p;
}

constexpr size_t kTileSmem = 128 + sizeof(StageSmem) + sizeof(TileSmem) + kBins1 * sizeof(unsigned);

// The walk kernel from this many pixels on (measured: 32 views of 1237 x 822 in
// 0.52 ms against 0.63 ms for the tile kernel; one such view in 0.087 against 0.051 ms).
constexpr long long kWalkMinPixels = 4LL << 20;

bool use_walk(const gsp_image_desc *imgs, int nv)
{
    long long px = 0;
    for (int v = 0; v < nv; ++v) px += (long long)imgs[v].width * imgs[v].height;
    return px >= kWalkMinPixels;
}

struct EdgeLayout {
    unsigned *hist1, *hist2, *sel, *cand_count, *med_bits, *bar;
    float *cand;
    float *kept;
    uint8_t *kmask;
    unsigned *kcount;
    PlainBufs plain;
    size_t bytes;
};

EdgeLayout edge_layout(void *ws, const gsp_image_desc *imgs, int nv, int mode, const EdgePlan &P)
{
    Carver c(ws);
    EdgeLayout L{};
    L.hist1 = c.take<unsigned>((size_t)nv * kBins1);
    L.hist2 = c.take<unsigned>((size_t)nv * kBins2);
    L.sel = c.take<unsigned>((size_t)nv * 4);
    L.cand_count = c.take<unsigned>(nv);
    L.med_bits = c.take<unsigned>(nv);
    L.bar = c.take<unsigned>(2);
    if (mode == GSP_EDGE_FUSED) {
        long long total = 0;
        for (int v = 0; v < nv; ++v)
            total = total > imgs[v].out_offset + (long long)imgs[v].width * imgs[v].height
                        ? total
                        : imgs[v].out_offset + (long long)imgs[v].width * imgs[v].height;
        L.cand = c.take<float>((size_t)total);
        if (use_walk(imgs, nv)) {
            L.kept = c.take<float>((size_t)P.items * kItemCols * P.rb);
            L.kmask = c.take<uint8_t>((size_t)P.items * (P.rb / 2) * 32);
            L.kcount = c.take<unsigned>((size_t)P.items);
        }
    } else {
        long long mw = 0, mh = 0;
        for (int v = 0; v < nv; ++v) {
            mw = mw > imgs[v].width ? mw : imgs[v].width;
            mh = mh > imgs[v].height ? mh : imgs[v].height;
        }
        // sized for the largest view, reused view after view
        size_t n8 = (size_t)(mw + 8) * (mh + 8), n6 = (size_t)(mw + 6) * (mh + 6);
        size_t nh = (size_t)(mw + 2) * (mh + 6), n2 = (size_t)(mw + 2) * (mh + 2);
        L.plain.I = c.take<int>(n8);
        L.plain.Sx = c.take<float>(n6);
        L.plain.Sy = c.take<float>(n6);
        L.plain.Hx = c.take<float>(nh);
        L.plain.Hy = c.take<float>(nh);
        L.plain.Gx = c.take<float>(n2);
        L.plain.Gy = c.take<float>(n2);
        L.plain.M = c.take<float>(n2);
        L.plain.hist = c.take<unsigned>(kBins1);
        L.plain.state = c.take<unsigned>(4);
    }
    L.bytes = c.size();
    return L;
}

// cuTensorMapEncodeTiled from the driver (looked up once through the runtime;
// null when the driver does not provide it: every view then reads directly).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map of a view's RGB bytes: uint8 [h][3 w] with the caller's row pitch,
// box kBoxW x kBoxH; out-of-range box parts read as zero (never used: the
// stencil indexes clamped coordinates).  False when TMA cannot stage the view.
bool encode_view_map(const gsp_image_desc &d, CUtensorMap *map)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    if ((reinterpret_cast<uintptr_t>(d.rgb) & 15) || (d.pitch_bytes & 15) || d.pitch_bytes >= (1LL << 40)) return false;
    const cuuint64_t dims[2] = {cuuint64_t(3) * cuuint64_t(d.width), cuuint64_t(d.height)};
    const cuuint64_t strides[1] = {cuuint64_t(d.pitch_bytes)};
    const cuuint32_t box[2] = {kBoxW, kBoxH};
    const cuuint32_t elem[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(d.rgb), dims, strides, box, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

gsp_status validate_edge(const gsp_image_desc *imgs, int nv, const gsp_edge_opts *o)
{
    if (!imgs || nv < 1) return GSP_ERR_INVALID_ARG;
    if (nv > GSP_MAX_VIEWS) return GSP_ERR_UNSUPPORTED;
    for (int v = 0; v < nv; ++v) {
        const gsp_image_desc &d = imgs[v];
        if (!d.rgb || d.width < 1 || d.height < 1 || d.pitch_bytes < 3LL * d.width || d.out_offset < 0)
            return GSP_ERR_INVALID_ARG;
        if ((long long)d.width * d.height > (1LL << 30)) return GSP_ERR_UNSUPPORTED;
    }
    if (o) {
        if (o->mode != GSP_EDGE_FUSED && o->mode != GSP_EDGE_PLAIN) return GSP_ERR_INVALID_ARG;
        if (o->use_custom_taps) {
            if (o->taps[0] != o->taps[4] || o->taps[1] != o->taps[3]) return GSP_ERR_INVALID_ARG;
        } else if (!(o->sigma > 0.f)) {
            return GSP_ERR_INVALID_ARG;
        }
    }
    return GSP_OK;
}

}  // namespace
}  // namespace gsp

using namespace gsp;

extern "C" void gsp_edge_opts_default(gsp_edge_opts *o)
{
    if (!o) return;
    *o = gsp_edge_opts{};
    o->mode = GSP_EDGE_FUSED;
    o->sigma = 1.0f;
    o->taps[0] = o->taps[4] = 0.f;
}

extern "C" size_t gsp_edge_map_workspace_size(const gsp_image_desc *imgs, int32_t nv, const gsp_edge_opts *opts)
{
    gsp_edge_opts o;
    gsp_edge_opts_default(&o);
    if (opts) o = *opts;
    if (validate_edge(imgs, nv, &o) != GSP_OK) return 0;
    return edge_layout(nullptr, imgs, nv, o.mode, edge_plan(imgs, nv)).bytes;
}

extern "C" gsp_status gsp_edge_map(const gsp_image_desc *imgs, int32_t nv, float *E_out, float *median_out,
                                   uint8_t *nms_mask_out, const gsp_edge_opts *opts, void *ws,
                                   size_t ws_bytes, int32_t *dev_status, gsp_stream_t stream)
{
    gsp_edge_opts o;
    gsp_edge_opts_default(&o);
    if (opts) o = *opts;
    gsp_status st = validate_edge(imgs, nv, &o);
    if (st != GSP_OK) return st;
    if (!E_out || !median_out || !dev_status) return GSP_ERR_INVALID_ARG;
    const EdgePlan P = edge_plan(imgs, nv);
    if (P.items >= (1LL << 31)) return GSP_ERR_UNSUPPORTED;
    EdgeLayout L = edge_layout(nullptr, imgs, nv, o.mode, P);
    st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = edge_layout(ws, imgs, nv, o.mode, P);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    const bool walk = o.mode == GSP_EDGE_FUSED && use_walk(imgs, nv);
    float w0, w1, w2;
    fill_taps(o, w0, w1, w2);
    const long long spin = o.spin_limit > 0 ? o.spin_limit : kDefaultSpinLimit;

    // histograms, candidate counters, medians and barrier state start at zero
    size_t zero_bytes = reinterpret_cast<char *>(L.bar + 2) - reinterpret_cast<char *>(L.hist1);
    GSP_CUDA_TRY(cudaMemsetAsync(L.hist1, 0, zero_bytes, s));

    int dev = 0;
    GSP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GSP_ERR_UNSUPPORTED;
    cudaLaunchAttribute coop[1];
    coop[0].id = cudaLaunchAttributeCooperative;
    coop[0].val.cooperative = 1;

    if (walk) {
        EdgeArgs a{};
        int items = 0;
        for (int v = 0; v < nv; ++v) {
            EdgeView &V = a.v[v];
            V.rgb = imgs[v].rgb;
            V.pitch = imgs[v].pitch_bytes;
            V.out_off = imgs[v].out_offset;
            V.w = imgs[v].width;
            V.h = imgs[v].height;
            V.groups = int(div_up(V.w, kItemCols));
            V.bands = int(div_up(V.h, P.rb));
            V.item_base = items;
            items += V.groups * V.bands;
        }
        a.nviews = nv;
        a.total_items = items;
        a.rb = P.rb;
        a.w0 = w0; a.w1 = w1; a.w2 = w2;
        a.E = E_out;
        a.mask = nms_mask_out;
        a.median_out = median_out;
        a.hist1 = L.hist1;
        a.hist2 = L.hist2;
        a.sel = L.sel;
        a.cand_count = L.cand_count;
        a.cand = L.cand;
        a.med_bits = L.med_bits;
        a.kept = L.kept;
        a.kmask = L.kmask;
        a.kcount = L.kcount;
        a.bar = L.bar;
        a.status = dev_status;
        a.spin_limit = spin;
        a.expire = o.test_expire & 1;
        int per_sm = 0;
        GSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_walk_kernel, WNT, 0));
        if (per_sm < 1) return GSP_ERR_UNSUPPORTED;
        if (o.blocks_per_sm > 0 && per_sm > o.blocks_per_sm) per_sm = o.blocks_per_sm;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(num_sms() * (per_sm < kWalkBlocksPerSM ? per_sm : kWalkBlocksPerSM));
        cfg.blockDim = dim3(WNT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = coop;
        cfg.numAttrs = 1;
        stage_begin("edge_fused", s);
        GSP_CUDA_TRY(cudaLaunchKernelEx(&cfg, edge_walk_kernel, a));
        stage_end("edge_fused", s);
        note_launches(2);
        return GSP_OK;
    }

    // the tile kernel (fused mode, small batches); its views also serve the plain path
    TileArgs a{};
    int tiles = 0;
    for (int v = 0; v < nv; ++v) {
        TileView &V = a.v[v];
        V.rgb = imgs[v].rgb;
        V.pitch = imgs[v].pitch_bytes;
        V.out_off = imgs[v].out_offset;
        V.w = imgs[v].width;
        V.h = imgs[v].height;
        V.tiles_x = int(div_up(V.w, TW));
        V.ntiles = V.tiles_x * int(div_up(V.h, TH));
        V.tile_base = tiles;
        tiles += V.ntiles;
        V.tma = o.mode == GSP_EDGE_FUSED && encode_view_map(imgs[v], &a.tmap[v]) ? 1 : 0;
    }
    a.nviews = nv;
    a.total_tiles = tiles;
    a.w0 = w0; a.w1 = w1; a.w2 = w2;
    a.E = E_out;
    a.mask = nms_mask_out;
    a.median_out = median_out;
    a.hist1 = L.hist1;
    a.hist2 = L.hist2;
    a.sel = L.sel;
    a.cand_count = L.cand_count;
    a.cand = L.cand;
    a.med_bits = L.med_bits;
    a.bar = L.bar;
    a.status = dev_status;
    a.spin_limit = spin;
    a.expire = o.test_expire & 3;

    if (o.mode == GSP_EDGE_FUSED) {
        static bool attr_set[kMaxDevices] = {false};
        if (!attr_set[dev]) {
            GSP_CUDA_TRY(cudaFuncSetAttribute(edge_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(kTileSmem)));
            attr_set[dev] = true;
        }
        int per_sm = 0;
        GSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_tile_kernel, NT, kTileSmem));
        if (per_sm < 1) return GSP_ERR_UNSUPPORTED;
        if (o.blocks_per_sm > 0 && per_sm > o.blocks_per_sm) per_sm = o.blocks_per_sm;
        int grid = per_sm * num_sms();
        if (grid > tiles) grid = tiles;
        if (grid < nv && nv <= per_sm * num_sms()) grid = nv;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = kTileSmem;
        cfg.stream = s;
        cfg.attrs = coop;
        cfg.numAttrs = 1;
        stage_begin("edge_fused", s);
        GSP_CUDA_TRY(cudaLaunchKernelEx(&cfg, edge_tile_kernel, a));
        stage_end("edge_fused", s);
        note_launches(2);
        return GSP_OK;
    }

    // plain: one launch per stage, view after view
    const PlainBufs &PB = L.plain;
    stage_begin("edge_plain", s);
    for (int v = 0; v < nv; ++v) {
        const TileView &V = a.v[v];
        long long n8 = (long long)(V.w + 8) * (V.h + 8), n6 = (long long)(V.w + 6) * (V.h + 6);
        long long nh = (long long)(V.w + 2) * (V.h + 6), n2 = (long long)(V.w + 2) * (V.h + 2);
        long long np = (long long)V.w * V.h;
        plain_luma<<<div_up(n8, 256), 256, 0, s>>>(V, PB.I);
        plain_sobel<<<div_up(n6, 256), 256, 0, s>>>(V, PB.I, PB.Sx, PB.Sy);
        plain_hblur<<<div_up(nh, 256), 256, 0, s>>>(V, PB.Sx, PB.Sy, PB.Hx, PB.Hy, w0, w1, w2);
        plain_vblur_mag<<<div_up(n2, 256), 256, 0, s>>>(V, PB.Hx, PB.Hy, PB.Gx, PB.Gy, PB.M, w0, w1, w2);
        plain_nms<<<div_up(np, 256), 256, 0, s>>>(V, PB.Gx, PB.Gy, PB.M, E_out, nms_mask_out);
        const int shifts[3] = {kShift1, kShift2, 0}, bins[3] = {kBins1, kBins2, kBins3};
        unsigned hist_blocks = div_up(np, 256 * 8);
        if (hist_blocks > 4u * num_sms()) hist_blocks = 4u * num_sms();
        for (int pass = 0; pass < 3; ++pass) {
            GSP_CUDA_TRY(cudaMemsetAsync(PB.hist, 0, kBins1 * sizeof(unsigned), s));
            plain_hist<<<hist_blocks, 256, 0, s>>>(E_out + V.out_off, np, shifts[pass], bins[pass], pass, PB.state,
                                                   PB.hist);
            plain_select<<<1, NT, 0, s>>>(PB.hist, bins[pass], shifts[pass], pass, PB.state, L.med_bits + v,
                                          median_out + v);
        }
        plain_normalise<<<div_up(np, 256), 256, 0, s>>>(V, E_out, L.med_bits + v);
    }
    stage_end("edge_plain", s);
    note_launches(1 + 15 * nv);
    GSP_LAUNCH_CHECK();
    return GSP_OK;
}
