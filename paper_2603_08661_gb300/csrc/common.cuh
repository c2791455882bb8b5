// Shared internals of libgsp: status reporting, workspace carving, launch
// helpers and a bounded grid barrier for the persistent kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsp.h"

namespace gsp {

constexpr int kTile = GSP_TILE;           // splatting tile edge (pixels)
constexpr int kTilePix = kTile * kTile;   // pixels per tile = threads per composite block

// Host-side record of the last CUDA error (per host thread).
void note_cuda_error(cudaError_t e);

// Instrumentation: launch counter, an NVTX range per stage (pushed by
// stage_begin, popped by stage_end) and the armed stage timer.
void note_launches(int n);
void stage_begin(const char *stage, cudaStream_t s);
void stage_end(const char *stage, cudaStream_t s);

#define GSP_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            gsp::note_cuda_error(_e);                        \
            return GSP_ERR_CUDA;                             \
        }                                                    \
    } while (0)

#define GSP_LAUNCH_CHECK() GSP_CUDA_TRY(cudaGetLastError())

// Device: record the first error code.
__device__ __forceinline__ void set_status(int32_t *st, int32_t code)
{
    atomicCAS(st, 0, code);
}

// Bounds-checked build (compiled with -DGSP_DEBUG, libgsp_debug.so): every index
// guarded by GSP_BOUND is compared with its bound before the access; an index
// out of bounds records GSP_ERR_CAPACITY in the status word and the access is
// skipped (nothing traps).  The release build compiles the guard away.
__device__ __forceinline__ bool bound_ok(unsigned long long i, unsigned long long n, int32_t *status)
{
    if (i < n) return true;
    if (status) set_status(status, GSP_ERR_CAPACITY);
    return false;
}
#ifdef GSP_DEBUG
#define GSP_BOUND(idx, bound, status) \
    gsp::bound_ok(static_cast<unsigned long long>(idx), static_cast<unsigned long long>(bound), (status))
#else
#define GSP_BOUND(idx, bound, status) true
#endif

// Bump allocator over a caller workspace; the same code sizes and carves.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t size() const { return (off + 255) & ~size_t(255); }
};

inline gsp_status check_workspace(const void *ws, size_t have, size_t need)
{
    if (need == 0) return GSP_OK;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || have < need) return GSP_ERR_WORKSPACE;
    return GSP_OK;
}

constexpr int kMaxDevices = 64;

// SM count of the current device (looked up once per device).
inline int num_sms()
{
    static int n[kMaxDevices] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) dev = 0;
    if (!n[dev]) {
        int c = 0;
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        n[dev] = c > 0 ? c : 1;
    }
    return n[dev];
}

inline unsigned div_up(long long a, long long b) { return static_cast<unsigned>((a + b - 1) / b); }

// Grid-wide barrier for co-resident (cooperatively launched) blocks.
// bar[0] counts arrivals, bar[1] is the generation.  Every wait polls at
// most spin_limit times; on expiry it records GSP_ERR_TIMEOUT and returns
// false, and the caller leaves the kernel.
// withhold (a test hook): the last block to arrive resets the count but does
// not open the barrier and leaves with GSP_ERR_TIMEOUT, so every other block's
// wait runs out - a flag that nothing sets.  The barrier state stays
// consistent (count 0, generation unchanged).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, long long spin_limit,
                                             int32_t *status, bool withhold = false)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            if (withhold) {
                set_status(status, GSP_ERR_TIMEOUT);
                ok = 0;
            } else {
                atomicAdd(bar + 1, 1u);
            }
        } else {
            long long polls = 0;
            while (*vgen == gen) {
                if (++polls > spin_limit || *(volatile int32_t *)status == GSP_ERR_TIMEOUT) {
                    set_status(status, GSP_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

constexpr long long kDefaultSpinLimit = 1ll << 23;

// ---- bulk asynchronous copies (TMA, 1-D) into shared memory, completed on an mbarrier
//
// One thread initialises the barrier, arms it with the byte count and issues
// the copies; every thread then waits on the barrier's phase.  A copy needs
// 16-byte aligned global and shared addresses and a size that is a multiple
// of 16 bytes.  The wait is bounded: after `limit` polls it gives up and the
// caller reports GSP_ERR_TIMEOUT (a copy that never lands is a bug, not a
// state to wait out).

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase, long long limit)
{
    for (long long i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace gsp
