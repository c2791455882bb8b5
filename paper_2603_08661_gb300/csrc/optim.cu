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
};

// blockIdx.y: the group.  Elements [0, N * row_len) of the flat group are
// updated with one FMA each (theta + (-lr) * grad, one rounding).
__global__ void __launch_bounds__(256) sgd_kernel(const __grid_constant__ SgdArgs a, const int32_t *count, float lr)
{
    const int grp = blockIdx.y;
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

}  // namespace
}  // namespace gsp

using namespace gsp;

extern "C" gsp_status gsp_sgd_step(const gsp_gaussians *g, float *grad_means, float *grad_log_scales,
                                   float *grad_quats, float *grad_opacity_logits, float *grad_sh, float lr,
                                   gsp_stream_t stream)
{
    if (!g || !g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh || !g->count)
        return GSP_ERR_INVALID_ARG;
    if (!grad_means || !grad_log_scales || !grad_quats || !grad_opacity_logits || !grad_sh)
        return GSP_ERR_INVALID_ARG;
    if (g->capacity < 1 || g->sh_degree < 0 || g->sh_degree > 3 || !(lr == lr)) return GSP_ERR_INVALID_ARG;
    const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
    SgdArgs a;
    float *ps[5] = {g->means, g->log_scales, g->quats, g->opacity_logits, g->sh};
    float *gs[5] = {grad_means, grad_log_scales, grad_quats, grad_opacity_logits, grad_sh};
    const int rl[5] = {3, 3, 4, 1, 3 * K};
    long long most = 0;
    for (int k = 0; k < 5; ++k) {
        a.p[k] = ps[k];
        a.g[k] = gs[k];
        a.row_len[k] = rl[k];
        a.vec4[k] = ((reinterpret_cast<uintptr_t>(ps[k]) | reinterpret_cast<uintptr_t>(gs[k])) & 15) == 0;
        most = std::max(most, (long long)g->capacity * rl[k]);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const unsigned blocks = unsigned(std::min<long long>(div_up(most / 4 + 1, 256), 8LL * num_sms()));
    stage_begin("sgd", s);
    sgd_kernel<<<dim3(blocks, 5), 256, 0, s>>>(a, g->count, lr);
    stage_end("sgd", s);
    note_launches(1);
    GSP_LAUNCH_CHECK();
    return GSP_OK;
}
