// Delay quantisation in FP64 (create time only).
//
// tau_ij = |x_i - x_j| / s_ij   (Eq. delaydist, Sec. 3.2.1; the general form
// D(x_i, x_j, Gamma_ij) >= 0 is Eq. gendelay, Sec. 2), in whole steps of dt:
//   d = sqrt(sum_k (x_i,k - x_j,k)^2)   summed in axis order
//   D = max(1, llround(d / (s * dt)))    half away from zero; a delay below half
//                                        a step is clamped to one step (an explicit
//                                        step cannot use a same-step value)
// Every operation is an explicitly rounded IEEE FP64 intrinsic, so no multiply-add
// is ever contracted and the table is the same on every machine that evaluates
// the same expression in the same order.
#include "internal.cuh"

namespace gn {
namespace {

__global__ void k_delay(int64_t n_edges, int32_t dim, const double *__restrict__ pos,
                        const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                        const double *__restrict__ speed, double speed_scalar, double dt_ms,
                        int32_t *__restrict__ delay, uint8_t *__restrict__ clamped)
{
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n_edges;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = src[e], j = dst[e];
        double sum = 0.0;
        for (int k = 0; k < dim; ++k) {
            const double diff = __dsub_rn(pos[i * dim + k], pos[j * dim + k]);
            sum = __dadd_rn(sum, __dmul_rn(diff, diff));
        }
        const double dist = __dsqrt_rn(sum);
        const double s = speed ? speed[e] : speed_scalar;
        const double q = __ddiv_rn(dist, __dmul_rn(s, dt_ms));
        long long d = llround(q);
        uint8_t cl = 0;
        if (d < 1) {
            d = 1;
            cl = 1;
        }
        if (d > 2147483647LL) d = 2147483647LL;  // reported as out of range by the host
        delay[e] = static_cast<int32_t>(d);
        clamped[e] = cl;
    }
}

}  // namespace

cudaError_t launch_delay(int64_t n_edges, int32_t dim, const double *pos, const int32_t *src,
                         const int32_t *dst, const double *speed, double speed_scalar, double dt_ms,
                         int32_t *delay, uint8_t *clamped, cudaStream_t s)
{
    if (n_edges <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n_edges + threads - 1) / threads;
    if (blocks > 148 * 64) blocks = 148 * 64;
    k_delay<<<static_cast<int>(blocks), threads, 0, s>>>(n_edges, dim, pos, src, dst, speed, speed_scalar,
                                                       dt_ms, delay, clamped);
    return cudaGetLastError();
}

}  // namespace gn
