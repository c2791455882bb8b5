// Edge-score selection and Long-Axis-Split (paper Sec. 2.2, Alg. 1 and Alg. 2).
//
// Selection: exact top-k in five launches that wait on nothing (so that they
// can interleave with other work).  Scores map to order-preserving 32-bit
// keys; the k-th largest key is found by a 3-digit radix select (11 + 11 + 10
// bits, one launch per digit counting into global histograms, every block of
// the next launch picking the same digit from the counts), every key above it
// is taken, and the ties at it are taken in ascending index order (ranks from
// a block scan plus the tie counts of the lower blocks; skipped when every
// tie is taken).
//
// Split: the selected Gaussians are ranked in index order by the same kind
// of scan; one thread per selected Gaussian applies Alg. 1: the long axis l
// is the argmax of the log-scales, the offset is k_off * exp(s_l) along
// column l of R read as entries l, l+3, l+6 of the row-major matrix (Alg. 2),
// the scales move in log space and the opacity in logit space.  Child 0
// replaces the parent; child 1 is appended at slot N + rank.  The capacity
// is checked on the device before anything is written.
#include <algorithm>

#include "common.cuh"

namespace gsp {
namespace {

constexpr int kThreads = 256, kPerThread = 4, kBlockItems = kThreads * kPerThread;
constexpr int kSelBins = 2048;

__device__ __forceinline__ unsigned order_key(float f)
{
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Block-local exclusive scan of per-thread counts; returns the block total.
__device__ unsigned block_scan(unsigned x, unsigned *excl)
{
    __shared__ unsigned wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned base = 0, tot = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
        if (w < wid) base += wsum[w];
        tot += wsum[w];
    }
    __syncthreads();
    *excl = base + inc - x;
    return tot;
}

struct MaskFlag {
    const uint8_t *mask;
    __device__ bool operator()(long long i) const { return mask[i] != 0; }
};

template <class F>
__global__ void __launch_bounds__(kThreads) flag_block_sums(F f, const int32_t *count, unsigned *sums)
{
    const long long n = *count;
    const long long b0 = (long long)blockIdx.x * kBlockItems;
    if (b0 >= n) return;
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        long long i = b0 + threadIdx.x * kPerThread + j;
        if (i < n && f(i)) ++c;
    }
    unsigned ex;
    unsigned tot = block_scan(c, &ex);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of the block sums (one block); total goes to sums[nblocks].
__global__ void __launch_bounds__(kThreads) scan_block_sums(const int32_t *count, unsigned *sums)
{
    __shared__ unsigned carry;
    const long long n = *count;
    const int nb = int((n + kBlockItems - 1) / kBlockItems);
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += kThreads) {
        int b = b0 + threadIdx.x;
        unsigned x = b < nb ? sums[b] : 0u;
        unsigned ex;
        unsigned tot = block_scan(x, &ex);
        unsigned c0 = carry;
        __syncthreads();
        if (b < nb) sums[b] = c0 + ex;
        if (threadIdx.x == 0) carry = c0 + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

struct TopkArgs {
    const float *scores;
    const int32_t *count;
    long long cap, k;
    uint8_t *mask;
    int32_t *selected_out;
    unsigned *hist;  // [3][kSelBins] digit counts of the three passes (zeroed before the launches)
    unsigned *sums;  // [grid] tie counts of the blocks' index ranges
    unsigned *state; // [4][4] the selection state after each stage (kk, prefix, remaining, eq)
    int32_t *status;
    // gradient-threshold masking (all three, or gsum == nullptr for none): Gaussian i
    // is a candidate when gcnt[i] > 0 and gsum[i] / gcnt[i] >= tau (FP32)
    const float *gsum;
    const int32_t *gcnt;
    float tau;
    unsigned *ncand;  // candidate count (zeroed before the launch)
    // importance sampling (expv != nullptr): Gaussian i with score > 0 rings at
    // expv[i] / score[i] (Exp(1) variates given by the caller); the k earliest
    // are taken, i.e. the k largest keys -expv[i] / score[i]
    const float *expv;
    long long budget;  // > 0: at most budget - N selected (the room left under a Gaussian budget)
};

__device__ __forceinline__ bool is_candidate(const TopkArgs &a, long long i)
{
    if (a.expv && !(a.scores[i] > 0.f)) return false;
    if (!a.gsum) return true;
    const int32_t c = a.gcnt[i];
    return c > 0 && __fdiv_rn(a.gsum[i], float(c)) >= a.tau;
}

// The value whose k largest are selected (for a candidate).
__device__ __forceinline__ float select_value(const TopkArgs &a, long long i)
{
    return a.expv ? -__fdiv_rn(a.expv[i], a.scores[i]) : a.scores[i];
}

// Block-wide pick of the digit that holds the rem-th largest key, from the
// counts hist[0 .. NB) (the top digit first): thread t owns the NB / kThreads
// digits [NB - (t+1) per, NB - t per), loaded at once and kept in registers;
// a scan of the owners' sums finds the owner, which walks its digits.
// Returns the digit; *above = keys in higher digits, *in_bin = keys in it.
template <int NB>
__device__ int pick_digit(const unsigned *hist, unsigned rem, unsigned *above, unsigned *in_bin)
{
    constexpr int per = NB / kThreads;
    __shared__ unsigned wsum[kThreads / 32];
    __shared__ int s_bin;
    __shared__ unsigned s_above, s_in;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned cnt[per];
    unsigned seg = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        cnt[q] = __ldcg(hist + NB - 1 - (threadIdx.x * per + q));
        seg += cnt[q];
    }
    unsigned inc = seg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    if (threadIdx.x == 0) s_bin = -1;
    __syncthreads();
    unsigned base = 0;
    for (int w = 0; w < wid; ++w) base += wsum[w];
    const unsigned before = base + inc - seg;
    if (before < rem && rem <= before + seg) {
        unsigned acc = before;
#pragma unroll
        for (int q = 0; q < per; ++q) {
            if (acc + cnt[q] >= rem) {
                s_bin = NB - 1 - (threadIdx.x * per + q);
                s_above = acc;
                s_in = cnt[q];
                break;
            }
            acc += cnt[q];
        }
    }
    __syncthreads();
    const int b = s_bin;
    *above = s_above;
    *in_bin = s_in;
    __syncthreads();
    return b;
}

// The selection in five launches, one per step (no block waits for another:
// the kernels can interleave with other work on the GPU):
//   stage 0, 1, 2  counts of digit pass `stage` (11 + 11 + 10 bits, the top
//                  digit first) over the keys that match the digits picked so
//                  far, after picking (every block the same) the digit of the
//                  previous pass from its global counts
//   stage 3        the last pick; the ties' counts of every block's index range
//                  when only some of the ties at the k-th key are taken
//   stage 4        the mask: every key above the k-th, and the first
//                  `remaining` ties in ascending index order
// Block 0 of each stage keeps the state (kk, prefix, remaining, eq) for the next.
__host__ __device__ constexpr int sel_shift(int pass) { return pass == 0 ? 21 : pass == 1 ? 10 : 0; }
__host__ __device__ constexpr int sel_bits(int pass) { return pass == 2 ? 10 : 11; }

struct SelState {
    unsigned kk, prefix, remaining, eq;
};

template <int STAGE>
__global__ void __launch_bounds__(kThreads) topk_stage(TopkArgs a)
{
    __shared__ unsigned h[kSelBins];
    const int tid = threadIdx.x;
    const unsigned G = gridDim.x;
    const long long n = max(*a.count, 0);
    SelState st;
    if (STAGE == 0) {
        unsigned kk = a.k < 0 ? 0u : (a.k > n ? unsigned(n) : unsigned(a.k));
        if (a.budget > 0) kk = unsigned(min((long long)kk, max(a.budget - n, 0LL)));
        st = {kk, 0u, kk, 0u};
    } else {
        const unsigned *w = a.state + 4 * (STAGE - 1);
        st = {__ldcg(w), __ldcg(w + 1), __ldcg(w + 2), __ldcg(w + 3)};
    }
    if (STAGE >= 1 && STAGE <= 3) {  // the digit of pass STAGE - 1
        constexpr int pass = STAGE >= 1 && STAGE <= 3 ? STAGE - 1 : 0;
        if (pass == 0 && (a.gsum || a.expv)) {  // at most the candidates
            st.kk = min(st.kk, __ldcg(a.ncand));
            st.remaining = st.kk;
        }
        if (st.remaining > 0) {
            unsigned above, in_bin;
            const int b = pick_digit<1 << sel_bits(pass)>(a.hist + pass * kSelBins, st.remaining, &above, &in_bin);
            st.prefix |= unsigned(b) << sel_shift(pass);
            st.remaining -= above;
            st.eq = in_bin;
        }
    }
    if (STAGE <= 3 && blockIdx.x == 0 && tid == 0) {
        unsigned *w = a.state + 4 * STAGE;
        w[0] = st.kk;
        w[1] = st.prefix;
        w[2] = st.remaining;
        w[3] = st.eq;
    }
    if (STAGE <= 2) {
        constexpr int pass = STAGE <= 2 ? STAGE : 0;
        constexpr int shift = sel_shift(pass), nb = 1 << sel_bits(pass), hi = shift + sel_bits(pass);
        if (st.remaining == 0) return;
        unsigned *gh = a.hist + pass * kSelBins;
        for (int i = tid; i < nb; i += kThreads) h[i] = 0;
        __syncthreads();
        // (four keys per thread and step, loaded before any is counted)
        unsigned nc = 0;
        const long long stride = (long long)G * kThreads;
        for (long long i0 = blockIdx.x * (long long)kThreads + tid; i0 < n; i0 += 4 * stride) {
            bool cand[4];
            float val[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = i0 + u * stride;
                cand[u] = i < n && is_candidate(a, i);
                val[u] = cand[u] ? select_value(a, i) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!cand[u]) continue;
                ++nc;
                const unsigned key = order_key(val[u]);
                if (pass > 0 && (key >> hi) != (st.prefix >> hi)) continue;
                atomicAdd(&h[(key >> shift) & unsigned(nb - 1)], 1u);
            }
        }
        nc = __reduce_add_sync(0xffffffffu, nc);
        if (pass == 0 && (a.gsum || a.expv) && (tid & 31) == 0 && nc) atomicAdd(a.ncand, nc);
        __syncthreads();
        for (int i = tid; i < nb; i += kThreads)
            if (h[i]) atomicAdd(gh + i, h[i]);
        return;
    }
    // prefix = t, the kk-th largest key; the keys above it are taken, and
    // `remaining` of the eq keys equal to it, in ascending index order
    const unsigned kk = st.kk, prefix = st.prefix, remaining = st.remaining;
    const bool rank_ties = kk > 0 && remaining < st.eq;
    const long long chunk = (a.cap + G - 1) / G;
    const long long b0 = min((long long)blockIdx.x * chunk, a.cap), b1 = min(b0 + chunk, a.cap);
    if (STAGE == 3) {
        if (!rank_ties) return;
        unsigned c = 0;
        const long long e = min(b1, n);
        for (long long i0 = b0 + tid; i0 < e; i0 += 4 * kThreads) {
            bool t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = i0 + u * kThreads;
                t[u] = i < e && is_candidate(a, i) && order_key(select_value(a, i)) == prefix;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) c += t[u];
        }
        unsigned ex;
        const unsigned tot = block_scan(c, &ex);
        if (tid == 0) a.sums[blockIdx.x] = tot;
        return;
    }
    unsigned tie_base = 0;
    if (rank_ties) {
        unsigned lower = 0;
        for (unsigned q = tid; q < blockIdx.x; q += kThreads) lower += __ldcg(a.sums + q);
        unsigned ex;
        tie_base = block_scan(lower, &ex);  // the block total: ties in the lower blocks' ranges
    }
    // mark the block's range, kPerThread consecutive items per thread per round
    for (long long r0 = b0; r0 < b1; r0 += kBlockItems) {
        bool tie[kPerThread], gt[kPerThread];
        unsigned c = 0;
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const long long i = r0 + tid * kPerThread + j;
            const unsigned key = (i < b1 && i < n) ? order_key(select_value(a, i)) : 0u;
            const bool live = i < b1 && i < n && kk > 0 && is_candidate(a, i);
            tie[j] = live && key == prefix;
            gt[j] = live && key > prefix;
            c += tie[j];
        }
        unsigned ex;
        const unsigned tot = block_scan(c, &ex);
        unsigned r = tie_base + ex;
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) {
            const long long i = r0 + tid * kPerThread + j;
            if (i >= b1) continue;
            a.mask[i] = gt[j] || (tie[j] && (!rank_ties || r < remaining));
            r += tie[j];
        }
        tie_base += tot;
    }
    if (a.selected_out && blockIdx.x == 0 && tid == 0) *a.selected_out = int32_t(kk);
}

struct LasArgs {
    float *means, *log_scales, *quats, *opac, *sh;
    int32_t *count;
    long long cap;
    int K;
    float k_off, log_long, log_other, beta;
    const uint8_t *mask;
    const unsigned *rank_off;  // block offsets; [nblocks] = total selected
    int32_t *src;              // [cap]: parent of appended child slot n + r
    int32_t *status;
};

__global__ void __launch_bounds__(kThreads) las_kernel(LasArgs a)
{
    const long long n = *a.count;
    const long long b0 = (long long)blockIdx.x * kBlockItems;
    if (b0 >= n) return;
    const int nb = int((n + kBlockItems - 1) / kBlockItems);
    const long long total = a.rank_off[nb];
    if (n + total > a.cap) return;  // reported by las_commit; nothing is written
    bool f[kPerThread];
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        long long i = b0 + threadIdx.x * kPerThread + j;
        f[j] = i < n && a.mask[i] != 0;
        c += f[j];
    }
    unsigned ex;
    block_scan(c, &ex);
    unsigned r = a.rank_off[blockIdx.x] + ex;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        if (!f[j]) continue;
        const long long i = b0 + threadIdx.x * kPerThread + j;
        const long long dst = n + r;
        ++r;
        if (!GSP_BOUND(dst, a.cap, a.status)) continue;
        float ls[3] = {a.log_scales[3 * i], a.log_scales[3 * i + 1], a.log_scales[3 * i + 2]};
        int l = 0;
        if (ls[1] > ls[l]) l = 1;
        if (ls[2] > ls[l]) l = 2;
        const float off = a.k_off * expf(ls[l]);
        float q[4] = {a.quats[4 * i], a.quats[4 * i + 1], a.quats[4 * i + 2], a.quats[4 * i + 3]};
        const float qi = __frsqrt_rn(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float w = q[0] * qi, x = q[1] * qi, y = q[2] * qi, z = q[3] * qi;
        // column l of the row-major rotation matrix: entries l, l + 3, l + 6 (Alg. 2)
        float cx, cy, cz;
        if (l == 0) {
            cx = 1.f - 2.f * (y * y + z * z); cy = 2.f * (x * y + w * z); cz = 2.f * (x * z - w * y);
        } else if (l == 1) {
            cx = 2.f * (x * y - w * z); cy = 1.f - 2.f * (x * x + z * z); cz = 2.f * (y * z + w * x);
        } else {
            cx = 2.f * (x * z + w * y); cy = 2.f * (y * z - w * x); cz = 1.f - 2.f * (x * x + y * y);
        }
        const float dx = cx * off, dy = cy * off, dz = cz * off;
        float nls[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) nls[k] = ls[k] + (k == l ? a.log_long : a.log_other);
        const float sig = 1.f / (1.f + expf(-a.opac[i]));
        const float p = a.beta * sig;
        const float nop = logf(p) - log1pf(-p);
        const float m0 = a.means[3 * i], m1 = a.means[3 * i + 1], m2 = a.means[3 * i + 2];
        // child 1 (appended)
        a.means[3 * dst] = m0 - dx; a.means[3 * dst + 1] = m1 - dy; a.means[3 * dst + 2] = m2 - dz;
        for (int k = 0; k < 3; ++k) a.log_scales[3 * dst + k] = nls[k];
        for (int k = 0; k < 4; ++k) a.quats[4 * dst + k] = q[k];
        a.opac[dst] = nop;
        a.src[dst - n] = int32_t(i);
        // child 0 (in place)
        a.means[3 * i] = m0 + dx; a.means[3 * i + 1] = m1 + dy; a.means[3 * i + 2] = m2 + dz;
        for (int k = 0; k < 3; ++k) a.log_scales[3 * i + k] = nls[k];
        a.opac[i] = nop;
    }
}

// SH rows of the appended children: one thread per (child, chunk), chunks of
// 16 bytes when the rows allow it (every copy independent: no per-row loop).
__global__ void __launch_bounds__(256) las_copy_sh(LasArgs a, int vec4)
{
    const long long n = *a.count;
    const int nb = int((n + kBlockItems - 1) / kBlockItems);
    const long long total = n > 0 ? a.rank_off[nb] : 0;
    if (n + total > a.cap) return;
    const int row = 3 * a.K;
    const int chunks = vec4 ? row / 4 : row;
    const long long work = total * chunks;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // four copies per thread and step, their parent indices and then their
    // source chunks loaded before any store (each copy is two dependent loads)
    constexpr int U = 4;
    for (long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; t0 < work; t0 += U * stride) {
        long long c[U], src[U];
        int q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long t = t0 + u * stride;
            c[u] = t < work ? t / chunks : -1;
            q[u] = t < work ? int(t - c[u] * chunks) : 0;
            src[u] = c[u] >= 0 ? (long long)a.src[c[u]] : -1;
        }
        if (vec4) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] >= 0 && GSP_BOUND(src[u], n, a.status))
                    v[u] = reinterpret_cast<const float4 *>(a.sh + (size_t)src[u] * row)[q[u]];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] >= 0 && src[u] >= 0 && src[u] < n)
                    reinterpret_cast<float4 *>(a.sh + (size_t)(n + c[u]) * row)[q[u]] = v[u];
        } else {
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] >= 0 && GSP_BOUND(src[u], n, a.status)) v[u] = a.sh[(size_t)src[u] * row + q[u]];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] >= 0 && src[u] >= 0 && src[u] < n) a.sh[(size_t)(n + c[u]) * row + q[u]] = v[u];
        }
    }
}

__global__ void las_commit(int32_t *count, long long cap, const unsigned *rank_off, int32_t *status)
{
    const long long n = *count;
    const int nb = int((n + kBlockItems - 1) / kBlockItems);
    const long long total = n > 0 ? rank_off[nb] : 0;
    if (n + total > cap) {
        set_status(status, GSP_ERR_CAPACITY);
        return;
    }
    *count = int32_t(n + total);
}

// [3][kSelBins] digit counts, the candidate count (zeroed before each
// selection), then the [4][4] stage states
constexpr int kTopkZeroWords = 3 * kSelBins + 1 + 16;

struct DensifyLayout {
    unsigned *hist;
    unsigned *ncand;
    unsigned *state;
    unsigned *sums;
    uint8_t *mask;
    int32_t *src;
    size_t bytes;
};

// The selection's scratch (shared by the workspace and the static array).
void carve_topk(Carver &c, long long cap, DensifyLayout &L)
{
    L.hist = c.take<unsigned>(kTopkZeroWords);
    L.ncand = L.hist + 3 * kSelBins;
    L.state = L.hist + 3 * kSelBins + 1;
    L.sums = c.take<unsigned>(div_up(cap, kBlockItems) + 1);
}

DensifyLayout densify_layout(void *ws, long long cap)
{
    Carver c(ws);
    DensifyLayout L{};
    carve_topk(c, cap, L);
    L.mask = c.take<uint8_t>((size_t)cap);
    L.src = c.take<int32_t>((size_t)cap);
    L.bytes = c.size();
    return L;
}

gsp_status enqueue_topk(const float *scores, const int32_t *count, long long cap, long long k, uint8_t *mask,
                        int32_t *selected_out, const DensifyLayout &L, int32_t *status, cudaStream_t s,
                        const float *gsum = nullptr, const int32_t *gcnt = nullptr, float tau = 0.f,
                        const float *expv = nullptr, long long budget = 0)
{
    // two blocks per SM, at most one per kBlockItems of capacity (the block sums are sized so)
    long long grid = 2LL * num_sms();
    grid = std::max(1LL, std::min(grid, (long long)div_up(cap, kBlockItems)));
    const TopkArgs a{scores, count, cap, k, mask, selected_out, L.hist, L.sums, L.state, status, gsum, gcnt, tau,
                     L.ncand, expv, budget};
    stage_begin("topk", s);
    GSP_CUDA_TRY(cudaMemsetAsync(L.hist, 0, (3 * kSelBins + 1) * sizeof(unsigned), s));
    const unsigned gb = unsigned(grid);
    topk_stage<0><<<gb, kThreads, 0, s>>>(a);
    topk_stage<1><<<gb, kThreads, 0, s>>>(a);
    topk_stage<2><<<gb, kThreads, 0, s>>>(a);
    topk_stage<3><<<gb, kThreads, 0, s>>>(a);
    topk_stage<4><<<gb, kThreads, 0, s>>>(a);
    stage_end("topk", s);
    note_launches(5);
    GSP_LAUNCH_CHECK();
    return GSP_OK;
}

}  // namespace
}  // namespace gsp

using namespace gsp;

extern "C" void gsp_las_params_paper(gsp_las_params *p)
{
    if (!p) return;
    p->k_off = 0.5f;
    p->long_factor = 0.5f;
    p->other_factor = 0.85f;
    p->beta = 0.6f;
}

extern "C" size_t gsp_las_workspace_size(int64_t capacity)
{
    if (capacity < 1) return 0;
    return densify_layout(nullptr, capacity).bytes;
}

extern "C" gsp_status gsp_topk_mask(const float *scores, const int32_t *count, int64_t capacity, int64_t k,
                                    uint8_t *mask_out, int32_t *selected_out, void *ws, size_t ws_bytes,
                                    int32_t *dev_status, gsp_stream_t stream)
{
    if (!scores || !count || !mask_out || !dev_status || capacity < 1 || capacity > (1LL << 30))
        return GSP_ERR_INVALID_ARG;
    DensifyLayout L = densify_layout(nullptr, capacity);
    gsp_status st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = densify_layout(ws, capacity);
    return enqueue_topk(scores, count, capacity, k, mask_out, selected_out, L, dev_status,
                        reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gsp_status gsp_topk_mask_gated(const float *scores, const float *pos_grad_sum,
                                          const int32_t *pos_grad_count, float threshold, const int32_t *count,
                                          int64_t capacity, int64_t k, uint8_t *mask_out, int32_t *selected_out,
                                          void *ws, size_t ws_bytes, int32_t *dev_status, gsp_stream_t stream)
{
    if (!scores || !pos_grad_sum || !pos_grad_count || !count || !mask_out || !dev_status || capacity < 1 ||
        capacity > (1LL << 30) || threshold != threshold)
        return GSP_ERR_INVALID_ARG;
    DensifyLayout L = densify_layout(nullptr, capacity);
    gsp_status st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = densify_layout(ws, capacity);
    return enqueue_topk(scores, count, capacity, k, mask_out, selected_out, L, dev_status,
                        reinterpret_cast<cudaStream_t>(stream), pos_grad_sum, pos_grad_count, threshold);
}

extern "C" gsp_status gsp_sample_mask(const float *scores, const float *exp_variates, const int32_t *count,
                                      int64_t capacity, int64_t k, uint8_t *mask_out, int32_t *selected_out,
                                      void *ws, size_t ws_bytes, int32_t *dev_status, gsp_stream_t stream)
{
    if (!scores || !exp_variates || !count || !mask_out || !dev_status || capacity < 1 ||
        capacity > (1LL << 30))
        return GSP_ERR_INVALID_ARG;
    DensifyLayout L = densify_layout(nullptr, capacity);
    gsp_status st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = densify_layout(ws, capacity);
    return enqueue_topk(scores, count, capacity, k, mask_out, selected_out, L, dev_status,
                        reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr, 0.f, exp_variates);
}

extern "C" gsp_status gsp_select_mask(const float *scores, const int32_t *count, int64_t capacity, int64_t k,
                                      const gsp_select_opts *opts, uint8_t *mask_out, int32_t *selected_out,
                                      void *ws, size_t ws_bytes, int32_t *dev_status, gsp_stream_t stream)
{
    if (!scores || !count || !mask_out || !dev_status || !opts || capacity < 1 || capacity > (1LL << 30))
        return GSP_ERR_INVALID_ARG;
    if (!opts->pos_grad_sum != !opts->pos_grad_count || opts->threshold != opts->threshold || opts->budget < 0)
        return GSP_ERR_INVALID_ARG;
    if (opts->pos_grad_sum && opts->exp_variates) return GSP_ERR_INVALID_ARG;  // gating is for the top-k
    DensifyLayout L = densify_layout(nullptr, capacity);
    gsp_status st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = densify_layout(ws, capacity);
    return enqueue_topk(scores, count, capacity, k, mask_out, selected_out, L, dev_status,
                        reinterpret_cast<cudaStream_t>(stream), opts->pos_grad_sum, opts->pos_grad_count,
                        opts->threshold, opts->exp_variates, opts->budget);
}

extern "C" gsp_status gsp_las_split(const gsp_gaussians *g, const uint8_t *mask, const float *scores, int64_t k,
                                    const gsp_las_params *p, void *ws, size_t ws_bytes, int32_t *dev_status,
                                    gsp_stream_t stream)
{
    if (!g || !g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh || !g->count || !p ||
        !dev_status)
        return GSP_ERR_INVALID_ARG;
    if (g->capacity < 1 || g->capacity > (1LL << 30) || g->sh_degree < 0 || g->sh_degree > 3)
        return GSP_ERR_INVALID_ARG;
    if (!mask && !scores) return GSP_ERR_INVALID_ARG;
    if (!(p->k_off >= 0.f) || !(p->long_factor > 0.f) || !(p->other_factor > 0.f) || !(p->beta > 0.f) ||
        !(p->beta <= 1.f))
        return GSP_ERR_INVALID_ARG;
    const long long cap = g->capacity;
    DensifyLayout L = densify_layout(nullptr, cap);
    gsp_status st = check_workspace(ws, ws_bytes, L.bytes);
    if (st != GSP_OK) return st;
    L = densify_layout(ws, cap);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!mask) {
        st = enqueue_topk(scores, g->count, cap, k, L.mask, nullptr, L, dev_status, s);
        if (st != GSP_OK) return st;
        mask = L.mask;
    }
    const unsigned nblk = div_up(cap, kBlockItems);
    MaskFlag mf{mask};
    stage_begin("las", s);
    flag_block_sums<<<nblk, kThreads, 0, s>>>(mf, g->count, L.sums);
    scan_block_sums<<<1, kThreads, 0, s>>>(g->count, L.sums);
    LasArgs a;
    a.means = g->means; a.log_scales = g->log_scales; a.quats = g->quats; a.opac = g->opacity_logits;
    a.sh = g->sh; a.count = g->count; a.cap = cap;
    a.K = (g->sh_degree + 1) * (g->sh_degree + 1);
    a.k_off = p->k_off;
    a.log_long = float(log(double(p->long_factor)));
    a.log_other = float(log(double(p->other_factor)));
    a.beta = p->beta;
    a.mask = mask;
    a.rank_off = L.sums;
    a.src = L.src;
    a.status = dev_status;
    las_kernel<<<nblk, kThreads, 0, s>>>(a);
    const int vec4 = (3 * a.K) % 4 == 0 && (reinterpret_cast<uintptr_t>(g->sh) & 15) == 0;
    las_copy_sh<<<4 * num_sms(), 256, 0, s>>>(a, vec4);
    las_commit<<<1, 1, 0, s>>>(g->count, cap, L.sums, dev_status);
    stage_end("las", s);
    note_launches(5);
    GSP_LAUNCH_CHECK();
    return GSP_OK;
}

// ------------------------------------------------- allocation-free top-k
//
// Some callers cannot allocate device memory at the time they call us:
// real-time loops that forbid allocation once they run, and host applications
// whose device memory is owned by their own allocator, where a plug-in may not
// take memory behind the host's back.  gsp_topk_mask_static
// serves them with the same selection as gsp_topk_mask, its scratch held in
// this file-scope device array instead of a caller workspace.  Every GPU that
// loads the library keeps the array until the process exits.

namespace gsp {
namespace {

constexpr long long kStaticTopkMaxCap = GSP_TOPK_STATIC_MAX_CAPACITY;
constexpr size_t kStaticTopkBytes = kTopkZeroWords * sizeof(unsigned) + 256 +
                                    sizeof(unsigned) * size_t((kStaticTopkMaxCap + kBlockItems - 1) / kBlockItems + 1) +
                                    256;

static __device__ __align__(256) unsigned char g_topk_scratch[kStaticTopkBytes];

static void *g_topk_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is only a stand-in for it).
gsp_status static_topk_scratch(void **out)
{
    int dev = 0;
    GSP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GSP_ERR_UNSUPPORTED;
    if (!g_topk_scratch_ptr[dev]) {
        void *p = nullptr;
        GSP_CUDA_TRY(cudaGetSymbolAddress(&p, g_topk_scratch));
        g_topk_scratch_ptr[dev] = p;
    }
    *out = g_topk_scratch_ptr[dev];
    return GSP_OK;
}

}  // namespace
}  // namespace gsp

extern "C" gsp_status gsp_topk_mask_static(const float *scores, const int32_t *count, int64_t capacity, int64_t k,
                                           uint8_t *mask_out, int32_t *selected_out, int32_t *dev_status,
                                           gsp_stream_t stream)
{
    if (!scores || !count || !mask_out || !dev_status || capacity < 1) return GSP_ERR_INVALID_ARG;
    if (capacity > kStaticTopkMaxCap) return GSP_ERR_INVALID_ARG;
    void *scratch = nullptr;
    gsp_status st = static_topk_scratch(&scratch);
    if (st != GSP_OK) return st;
    // same carving as a workspace, without the mask (the caller's output)
    Carver c(scratch);
    DensifyLayout L{};
    carve_topk(c, capacity, L);
    L.mask = nullptr;
    if (c.size() > kStaticTopkBytes) return GSP_ERR_UNSUPPORTED;
    return enqueue_topk(scores, count, capacity, k, mask_out, selected_out, L, dev_status,
                        reinterpret_cast<cudaStream_t>(stream));
}
