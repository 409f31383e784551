// Host entry points of the connectivity estimator: features on device buffers
// (k_est.cu), the learned estimator (k_mlp.cu) and the scores a mapping is judged
// by (area under the ROC curve, F1), computed on the host in FP64.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "runtime.h"

using gnrt::cuda_check;
using gnrt::fail;
using gnrt::guarded;

namespace {

void check_scores(const float *scores, const uint8_t *labels, int64_t n)
{
    if (n < 0 || (n > 0 && (!scores || !labels))) fail(GN_EINVAL, "bad score arrays");
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(scores[i])) fail(GN_EINVAL, "score %lld is not finite", (long long)i);
}

}  // namespace

extern "C" {

gn_status gn_xcorr_features(const float *traces, int64_t n_nodes, int32_t n_samples, const double *pos, int32_t dim,
                            int64_t n_pairs, const int32_t *src, const int32_t *dst, const double *radius,
                            double v_max, double sample_ms, float *features, float *score, void *cuda_stream)
{
    return guarded([&] {
        if (n_nodes < 0 || n_samples < 1 || n_pairs < 0 || dim < 1 || dim > 3) fail(GN_EINVAL, "bad sizes");
        if (!(v_max > 0.0) || !(sample_ms > 0.0)) fail(GN_EINVAL, "v_max and sample_ms must be positive");
        if (n_pairs > 0 && (!traces || !pos || !src || !dst || !radius || !features || !score))
            fail(GN_EINVAL, "a device pointer is NULL");
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        float *scratch = nullptr;
        const int64_t nf = std::max<int64_t>(1, gn::ncc_scratch_floats(n_nodes, n_samples));
        cuda_check(cudaMallocAsync(reinterpret_cast<void **>(&scratch), nf * sizeof(float), s), "cudaMallocAsync");
        cudaError_t e = gn::launch_ncc(traces, n_nodes, n_samples, scratch, pos, dim, n_pairs, src, dst, radius, v_max,
                                       sample_ms, features, score, s);
        cudaFreeAsync(scratch, s);
        cuda_check(e, "correlation kernel");
    });
}

gn_status gn_score_auroc(const float *scores, const uint8_t *labels, int64_t n, double *auroc)
{
    return guarded([&] {
        check_scores(scores, labels, n);
        if (!auroc) fail(GN_EINVAL, "auroc is NULL");
        // Mann-Whitney U with mid-ranks: AUROC = (R_pos - n_pos (n_pos + 1) / 2) / (n_pos n_neg)
        std::vector<int64_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return scores[a] < scores[b]; });
        double rank_pos = 0.0;
        int64_t n_pos = 0;
        for (int64_t i = 0; i < n;) {
            int64_t j = i;
            while (j < n && scores[order[j]] == scores[order[i]]) ++j;
            const double mid = 0.5 * static_cast<double>(i + 1 + j);  // mean of ranks i+1 .. j
            for (int64_t k = i; k < j; ++k)
                if (labels[order[k]]) {
                    rank_pos += mid;
                    ++n_pos;
                }
            i = j;
        }
        const int64_t n_neg = n - n_pos;
        *auroc = (n_pos == 0 || n_neg == 0)
                     ? NAN
                     : (rank_pos - 0.5 * static_cast<double>(n_pos) * static_cast<double>(n_pos + 1)) /
                           (static_cast<double>(n_pos) * static_cast<double>(n_neg));
    });
}

gn_status gn_score_f1(const float *scores, const uint8_t *labels, int64_t n, double threshold, double *f1)
{
    return guarded([&] {
        check_scores(scores, labels, n);
        if (!f1) fail(GN_EINVAL, "f1 is NULL");
        int64_t tp = 0, fp = 0, fn = 0;
        for (int64_t i = 0; i < n; ++i) {
            const bool pred = static_cast<double>(scores[i]) >= threshold;
            tp += pred && labels[i];
            fp += pred && !labels[i];
            fn += !pred && labels[i];
        }
        *f1 = (tp + fp + fn) ? 2.0 * tp / static_cast<double>(2 * tp + fp + fn) : 0.0;
    });
}

gn_status gn_score_best_f1(const float *scores, const uint8_t *labels, int64_t n, double *threshold, double *f1)
{
    return guarded([&] {
        check_scores(scores, labels, n);
        if (!threshold || !f1) fail(GN_EINVAL, "outputs are NULL");
        // sweep thresholds from the highest score down: "edge iff score >= s"
        std::vector<int64_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return scores[a] > scores[b]; });
        int64_t pos_total = 0;
        for (int64_t i = 0; i < n; ++i) pos_total += labels[i] ? 1 : 0;
        int64_t tp = 0, fp = 0;
        double best = -1.0, best_thr = n ? scores[order[0]] : 0.0;
        for (int64_t i = 0; i < n; ++i) {
            tp += labels[order[i]] ? 1 : 0;
            fp += labels[order[i]] ? 0 : 1;
            if (i + 1 < n && scores[order[i + 1]] == scores[order[i]]) continue;  // ties go together
            const int64_t fn = pos_total - tp;
            const double f = 2.0 * tp / static_cast<double>(std::max<int64_t>(1, 2 * tp + fp + fn));
            if (f > best) {
                best = f;
                best_thr = scores[order[i]];
            }
        }
        *threshold = best_thr;
        *f1 = std::max(best, 0.0);
    });
}

}  // extern "C"
