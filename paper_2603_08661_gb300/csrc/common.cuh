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

// Instrumentation: launch counter and the armed stage timer.
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

inline int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

inline unsigned div_up(long long a, long long b) { return static_cast<unsigned>((a + b - 1) / b); }

// Grid-wide barrier for co-resident (cooperatively launched) blocks.
// bar[0] counts arrivals, bar[1] is the generation.  Every wait polls at
// most spin_limit times; on expiry it records GSP_ERR_TIMEOUT and returns
// false, and the caller leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, long long spin_limit,
                                             int32_t *status)
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
            atomicAdd(bar + 1, 1u);
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

}  // namespace gsp
