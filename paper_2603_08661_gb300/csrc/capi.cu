// Status strings, the per-thread CUDA error record, the version query and the
// stage instrumentation: an NVTX range per stage of every call (host-side
// enqueue ranges named after the stage, for profilers that filter on them;
// free when no tool is attached) and the armed CUDA-event stage timer.
#include "common.cuh"

#include <nvtx3/nvToolsExt.h>
#include <string.h>

#include <vector>

namespace gsp {
static thread_local int32_t g_last_cuda_error = 0;
void note_cuda_error(cudaError_t e) { g_last_cuda_error = int32_t(e); }

static long long g_launches = 0;
void note_launches(int n) { g_launches += n; }

struct StageTimer {
    char name[32] = {0};
    std::vector<cudaEvent_t> ev;  // pairs
    int used = 0;
    bool open = false;
};
static StageTimer g_timer;

// Inside stream capture the events must become event-record nodes of the
// graph (external records), so that each replay records them.
static void record(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

void stage_begin(const char *stage, cudaStream_t s)
{
    nvtxRangePushA(stage);
    if (!g_timer.name[0] || strcmp(g_timer.name, stage) != 0) return;
    if (2 * (g_timer.used + 1) > int(g_timer.ev.size())) return;
    record(g_timer.ev[2 * g_timer.used], s);
    g_timer.open = true;
}

void stage_end(const char *stage, cudaStream_t s)
{
    nvtxRangePop();
    if (!g_timer.open || strcmp(g_timer.name, stage) != 0) return;
    record(g_timer.ev[2 * g_timer.used + 1], s);
    g_timer.used++;
    g_timer.open = false;
}
}  // namespace gsp

extern "C" int64_t gsp_kernel_launch_count(void) { return gsp::g_launches; }

extern "C" gsp_status gsp_stage_timer_arm(const char *stage, int32_t max_records)
{
    using gsp::g_timer;
    for (cudaEvent_t e : g_timer.ev) cudaEventDestroy(e);
    g_timer.ev.clear();
    g_timer.used = 0;
    g_timer.open = false;
    g_timer.name[0] = 0;
    if (!stage) return GSP_OK;
    if (strlen(stage) >= sizeof(g_timer.name) || max_records < 1 || max_records > 4096) return GSP_ERR_INVALID_ARG;
    g_timer.ev.resize(size_t(2) * max_records);
    for (auto &e : g_timer.ev) GSP_CUDA_TRY(cudaEventCreate(&e));
    strcpy(g_timer.name, stage);
    return GSP_OK;
}

extern "C" gsp_status gsp_stage_timer_read(float *total_ms, int32_t *occurrences)
{
    using gsp::g_timer;
    if (!total_ms || !occurrences) return GSP_ERR_INVALID_ARG;
    float sum = 0.f;
    for (int k = 0; k < g_timer.used; ++k) {
        GSP_CUDA_TRY(cudaEventSynchronize(g_timer.ev[2 * k + 1]));
        float ms = 0.f;
        GSP_CUDA_TRY(cudaEventElapsedTime(&ms, g_timer.ev[2 * k], g_timer.ev[2 * k + 1]));
        sum += ms;
    }
    *total_ms = sum;
    *occurrences = g_timer.used;
    return GSP_OK;
}

extern "C" const char *gsp_status_string(int32_t s)
{
    switch (s) {
    case GSP_OK: return "ok";
    case GSP_ERR_INVALID_ARG: return "invalid argument";
    case GSP_ERR_CUDA: return "CUDA runtime error";
    case GSP_ERR_CAPACITY: return "capacity exceeded (pairs or Gaussians); outputs not written";
    case GSP_ERR_TIMEOUT: return "grid barrier wait timed out";
    case GSP_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case GSP_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

extern "C" int32_t gsp_last_cuda_error(void) { return gsp::g_last_cuda_error; }

extern "C" int32_t gsp_version(void) { return 100; }
