// Connectivity-estimator kernels: trace export and lagged normalised
// cross-correlation features.
//
// Correlating the activity of two cells is the common way to map functional
// connections (Sec. 1); on geometric networks the signal of i reaches j after the
// delay |x_i - x_j| / s (Sec. 3.2.1, Eq. delaydist), so the features of a
// candidate pair i -> j are the correlations of y_i(t) with y_j(t + l) for 32
// lags l starting at the shortest geometric delay d / v_max, plus d / r_c.
#include "internal.cuh"

namespace gn {
namespace {

// Node-major traces from the observation rings of a batch: out[(node_off + j) * T + t]
// = obs[((first + t) mod cap) * N + j], one 32 x 32 tile per CTA (coalesced both ways).
__global__ void k_export_traces(const float *__restrict__ obs_pool, const ExportNet *__restrict__ nets,
                                int64_t first, int T, int64_t cap, float *__restrict__ out)
{
    __shared__ float tile[32][33];
    const ExportNet e = nets[blockIdx.z];
    const int j0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
    if (j0 >= e.n_nodes || t0 >= T) return;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int t = t0 + r, j = j0 + tx;
        if (t < T && j < e.n_nodes) tile[r][tx] = obs_pool[e.obs_off + ((first + t) % cap) * e.n_nodes + j];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r, t = t0 + tx;
        if (t < T && j < e.n_nodes) out[(e.node_off + j) * static_cast<int64_t>(T) + t] = tile[tx][r];
    }
}

// Per node (one warp): the trace centred on its own mean, a(t) = y(t) - m, and the
// prefix sums P1[t] = sum_{s<t} a(s), P2[t] = sum_{s<t} a(s)^2, t = 0..T, so any
// segment's first two moments are two lookups.
__global__ void k_trace_prefix(const float *__restrict__ X, int64_t M, int T, float *__restrict__ A,
                               float *__restrict__ P1, float *__restrict__ P2)
{
    const int64_t node = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (node >= M) return;
    const float *x = X + node * T;
    float s = 0.0f;
    for (int t = lane; t < T; t += 32) s += x[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float m = s / static_cast<float>(T);
    float *a_out = A + node * T;
    float *p1 = P1 + node * (T + 1);
    float *p2 = P2 + node * (T + 1);
    if (lane == 0) {
        p1[0] = 0.0f;
        p2[0] = 0.0f;
    }
    float c1 = 0.0f, c2 = 0.0f;  // sums of the chunks before this one
    for (int t0 = 0; t0 < T; t0 += 32) {
        const int t = t0 + lane;
        const float a = t < T ? x[t] - m : 0.0f;
        if (t < T) a_out[t] = a;
        float q1 = a, q2 = a * a;  // inclusive scan over the chunk
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float u1 = __shfl_up_sync(0xffffffffu, q1, o);
            const float u2 = __shfl_up_sync(0xffffffffu, q2, o);
            if (lane >= o) {
                q1 += u1;
                q2 += u2;
            }
        }
        if (t < T) {
            p1[t + 1] = c1 + q1;
            p2[t + 1] = c2 + q2;
        }
        c1 += __shfl_sync(0xffffffffu, q1, 31);
        c2 += __shfl_sync(0xffffffffu, q2, 31);
    }
}

// One warp per candidate pair, lane k = lag l = l0 + k.  Over the overlap
// t < n = T - l of a = y_i(t) - m_i and b = y_j(t + l) - m_j the Pearson correlation
// of the two segments about their own means is
//   r = (S_ab - S_a S_b / n) / sqrt((S_aa - S_a^2 / n)(S_bb - S_b^2 / n)),
// 0 when either segment is constant.  S_a, S_aa come from node i's prefix sums at n,
// S_b, S_bb from node j's between l and T; only S_ab is summed here (the source
// trace read four samples at a time, the same words for every lane).  The distance
// and the first lag are FP64 in the order of their definition (d = sqrt(sum of
// squared coordinate differences), l0 = floor((d / v_max) / sample)), so the integer
// lag is the same as the oracle's.
__global__ void k_ncc(const float *__restrict__ A, const float *__restrict__ P1, const float *__restrict__ P2, int T,
                      const double *__restrict__ pos, int dim, int64_t P, const int *__restrict__ src,
                      const int *__restrict__ dst, const double *__restrict__ radius, double v_max, double sample_ms,
                      float *__restrict__ feat, float *__restrict__ score)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    const bool vec = (T & 3) == 0;
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32; p < P; p += warps) {
        const int64_t i = src[p], j = dst[p];
        double s2 = 0.0;
        for (int k = 0; k < dim; ++k) {
            const double diff = __dsub_rn(pos[i * dim + k], pos[j * dim + k]);
            s2 = __dadd_rn(s2, __dmul_rn(diff, diff));
        }
        const double d = __dsqrt_rn(s2);
        const int l0 = static_cast<int>(floor(__ddiv_rn(__ddiv_rn(d, v_max), sample_ms)));
        const int lag = l0 + lane;
        const int n = T - lag;
        const float *ai = A + i * T;
        const float *bj = A + j * T + lag;
        float sab = 0.0f;
        const int tmax = T - l0;  // the longest overlap (lane 0)
        int t = 0;
        if (vec) {
            for (; t + 4 <= tmax; t += 4) {
                const float4 a4 = __ldg(reinterpret_cast<const float4 *>(ai + t));
                const float b0 = t < n ? __ldg(bj + t) : 0.0f;
                const float b1 = t + 1 < n ? __ldg(bj + t + 1) : 0.0f;
                const float b2 = t + 2 < n ? __ldg(bj + t + 2) : 0.0f;
                const float b3 = t + 3 < n ? __ldg(bj + t + 3) : 0.0f;
                sab = fmaf(a4.x, b0, sab);
                sab = fmaf(a4.y, b1, sab);
                sab = fmaf(a4.z, b2, sab);
                sab = fmaf(a4.w, b3, sab);
            }
        }
        for (; t < tmax; ++t)
            if (t < n) sab = fmaf(__ldg(ai + t), __ldg(bj + t), sab);
        float r = 0.0f;
        if (n >= 2) {
            const float *pi1 = P1 + i * (T + 1), *pi2 = P2 + i * (T + 1);
            const float *pj1 = P1 + j * (T + 1), *pj2 = P2 + j * (T + 1);
            const float sa = __ldg(pi1 + n), saa = __ldg(pi2 + n);
            const float sb = __ldg(pj1 + T) - __ldg(pj1 + lag), sbb = __ldg(pj2 + T) - __ldg(pj2 + lag);
            const float inv_n = 1.0f / static_cast<float>(n);
            const float cov = sab - sa * sb * inv_n;
            const float va = saa - sa * sa * inv_n;
            const float vb = sbb - sb * sb * inv_n;
            if (va > 0.0f && vb > 0.0f) r = cov * rsqrtf(va * vb);
        }
        feat[p * 33 + lane] = r;
        float mx = r;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            feat[p * 33 + 32] = static_cast<float>(__ddiv_rn(d, radius[p]));
            score[p] = mx;
        }
    }
}

}  // namespace

cudaError_t launch_export_traces(const float *obs_pool, const ExportNet *nets, int n_nets, int max_nodes,
                                 int64_t first, int T, int64_t cap, float *out, cudaStream_t s)
{
    if (n_nets <= 0 || T <= 0) return cudaSuccess;
    dim3 grid((max_nodes + 31) / 32, (T + 31) / 32, n_nets);
    k_export_traces<<<grid, dim3(32, 8), 0, s>>>(obs_pool, nets, first, T, cap, out);
    return cudaGetLastError();
}

cudaError_t launch_ncc(const float *X, int64_t M, int T, float *scratch, const double *pos, int dim, int64_t P,
                       const int *src, const int *dst, const double *radius, double v_max, double sample_ms,
                       float *feat, float *score, cudaStream_t s)
{
    float *A = scratch;
    float *P1 = A + M * T;
    float *P2 = P1 + M * (T + 1);
    if (M > 0) {
        k_trace_prefix<<<static_cast<unsigned>((M + 7) / 8), 256, 0, s>>>(X, M, T, A, P1, P2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (P <= 0) return cudaSuccess;
    int64_t blocks = (P + 7) / 8;
    if (blocks > 148 * 64) blocks = 148 * 64;
    k_ncc<<<static_cast<unsigned>(blocks), 256, 0, s>>>(A, P1, P2, T, pos, dim, P, src, dst, radius, v_max, sample_ms,
                                                         feat, score);
    return cudaGetLastError();
}

int64_t ncc_scratch_floats(int64_t M, int T) { return M * T + 2 * M * (T + 1); }

}  // namespace gn
