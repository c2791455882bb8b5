// Plain SGD on the live rows of every parameter group, one launch.  The
// paper does not describe its optimiser; this is the update of the
// device-resident densification loop (theta <- theta - lr * grad).
#include <algorithm>

#include "common.cuh"

namespace gsp {
namespace {

struct SgdArgs {
    float *p[5];
    const float *g[5];
    int row_len[5];  // floats per Gaussian in each group
    int vec4[5];     // parameter and gradient 16-byte aligned: float4 body
    // learning rates: lr_init[grp] when step is null, else the exponential
    // schedule lr_init * (lr_final / lr_init)^(min(t, steps) / steps) at t = *step
    float lr_init[5], lr_final[5];
    int steps;
    const int32_t *step;
};

__device__ __forceinline__ float scheduled_lr(const SgdArgs &a, int grp)
{
    const float l0 = a.lr_init[grp], l1 = a.lr_final[grp];
    if (!a.step || l0 == l1) return l0;
    const int t = min(max(*a.step, 0), a.steps);
    return l0 * expf(logf(l1 / l0) * (float(t) / float(a.steps)));
}

// blockIdx.y: the group.  Elements [0, N * row_len) of the flat group are
// updated with one FMA each (theta + (-lr) * grad, one rounding).
__global__ void __launch_bounds__(256) sgd_kernel(const __grid_constant__ SgdArgs a, const int32_t *count)
{
    const int grp = blockIdx.y;
    const float lr = scheduled_lr(a, grp);
    float *p = a.p[grp];
    const float *g = a.g[grp];
    const long long n = (long long)max(*count, 0) * a.row_len[grp];
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a.vec4[grp]) {
        const long long n4 = n / 4;
        float4 *p4 = reinterpret_cast<float4 *>(p);
        const float4 *g4 = reinterpret_cast<const float4 *>(g);
        for (long long j = i; j < n4; j += stride) {
            float4 x = p4[j];
            const float4 d = g4[j];
            x.x = __fmaf_rn(-lr, d.x, x.x);
            x.y = __fmaf_rn(-lr, d.y, x.y);
            x.z = __fmaf_rn(-lr, d.z, x.z);
            x.w = __fmaf_rn(-lr, d.w, x.w);
            p4[j] = x;
        }
        for (long long j = 4 * n4 + i; j < n; j += stride) p[j] = __fmaf_rn(-lr, g[j], p[j]);
    } else {
        for (long long j = i; j < n; j += stride) p[j] = __fmaf_rn(-lr, g[j], p[j]);
    }
}

// The schedule's step counter advances once the step's updates are enqueued.
__global__ void advance_step(int32_t *step) { *step += 1; }

gsp_status enqueue_sgd(const gsp_gaussians *g, float *const grads[5], const float lr_init[5], const float lr_final[5],
                       int steps, int32_t *step, cudaStream_t s)
{
    if (!g || !g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh || !g->count)
        return GSP_ERR_INVALID_ARG;
    for (int k = 0; k < 5; ++k)
        if (!grads[k] || !(lr_init[k] == lr_init[k]) || !(lr_final[k] == lr_final[k])) return GSP_ERR_INVALID_ARG;
    if (g->capacity < 1 || g->sh_degree < 0 || g->sh_degree > 3) return GSP_ERR_INVALID_ARG;
    const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
    SgdArgs a;
    float *ps[5] = {g->means, g->log_scales, g->quats, g->opacity_logits, g->sh};
    const int rl[5] = {3, 3, 4, 1, 3 * K};
    long long most = 0;
    for (int k = 0; k < 5; ++k) {
        a.p[k] = ps[k];
        a.g[k] = grads[k];
        a.row_len[k] = rl[k];
        a.vec4[k] = ((reinterpret_cast<uintptr_t>(ps[k]) | reinterpret_cast<uintptr_t>(grads[k])) & 15) == 0;
        a.lr_init[k] = lr_init[k];
        a.lr_final[k] = lr_final[k];
        most = std::max(most, (long long)g->capacity * rl[k]);
    }
    a.steps = steps;
    a.step = step;
    const unsigned blocks = unsigned(std::min<long long>(div_up(most / 4 + 1, 256), 8LL * num_sms()));
    stage_begin("sgd", s);
    sgd_kernel<<<dim3(blocks, 5), 256, 0, s>>>(a, g->count);
    if (step) advance_step<<<1, 1, 0, s>>>(step);
    stage_end("sgd", s);
    note_launches(step ? 2 : 1);
    GSP_LAUNCH_CHECK();
    return GSP_OK;
}

}  // namespace
}  // namespace gsp

using namespace gsp;

extern "C" gsp_status gsp_sgd_step(const gsp_gaussians *g, float *grad_means, float *grad_log_scales,
                                   float *grad_quats, float *grad_opacity_logits, float *grad_sh, float lr,
                                   gsp_stream_t stream)
{
    float *const grads[5] = {grad_means, grad_log_scales, grad_quats, grad_opacity_logits, grad_sh};
    const float l[5] = {lr, lr, lr, lr, lr};
    return enqueue_sgd(g, grads, l, l, 1, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" gsp_status gsp_sgd_step_scheduled(const gsp_gaussians *g, float *grad_means, float *grad_log_scales,
                                             float *grad_quats, float *grad_opacity_logits, float *grad_sh,
                                             const gsp_lr_schedule *sched, int32_t *step, gsp_stream_t stream)
{
    if (!sched || !step || sched->steps < 1) return GSP_ERR_INVALID_ARG;
    for (int k = 0; k < 5; ++k)  // an exponential between two rates needs both positive
        if (sched->lr_init[k] != sched->lr_final[k] && !(sched->lr_init[k] > 0.f && sched->lr_final[k] > 0.f))
            return GSP_ERR_INVALID_ARG;
    float *const grads[5] = {grad_means, grad_log_scales, grad_quats, grad_opacity_logits, grad_sh};
    return enqueue_sgd(g, grads, sched->lr_init, sched->lr_final, sched->steps, step,
                       reinterpret_cast<cudaStream_t>(stream));
}
