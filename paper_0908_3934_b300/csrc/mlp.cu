// Host runtime of the learned estimator (gn_mlp_* in include/geonet.h): an MLP
// in -> 256 -> 256 -> 1 trained with the project's own forward, backward and
// AdamW kernels (k_mlp.cu) on device-resident batches.
//
// Parameters, gradients and Adam moments are packed FP32 buffers in one layout,
// [W1 (in x 256) | b1 | W2 (256 x 256) | b2 | w3 | b3], so AdamW is one
// elementwise launch; BF16 copies of W1 and W2 in the layouts the GEMMs read are
// refreshed after every update.
#include <algorithm>
#include <cmath>
#include <vector>

#include "runtime.h"

using gnrt::cuda_check;
using gnrt::DevArray;
using gnrt::DeviceGuard;
using gnrt::fail;
using gnrt::guarded;

namespace {
constexpr int H = gn::kMlpHidden;
constexpr int KP = gn::kMlpInPad;
constexpr int kChunk = 128;  // batch padding granularity and the smallest weight-gradient split
constexpr int kHeadRows = 64;
}  // namespace

struct gn_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int in_dim = 0;
    int max_bp = 0;  // workspace rows (multiple of 128)
    int64_t n_params = 0;
    int64_t off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_w3 = 0, off_b3 = 0;
    int64_t adam_t = 0;
    size_t bytes = 0;
    DevArray<float> params, grads, m, v;
    DevArray<uint16_t> W1t, W2t, W2b;                 // BF16 copies
    DevArray<uint16_t> Xb, H1, dH2, dH1;              // BF16 activations [max_bp][.]
    DevArray<uint16_t> XT, H1T, dH2T, dH1T;           // the same transposed, [.][Bp] (weight-gradient operands)
    DevArray<float> H2, p, part_w2, part_w1, part_head, part_b1, tmp_w1, tmp_head;
    DevArray<unsigned int> status;  // kStatusTimeout when a kernel's bounded wait gave up
    // replayed training epochs: batch cursor, bias-correction table, per-step losses
    DevArray<int64_t> ep_cursor;
    DevArray<float> ep_bc, ep_losses;
    cudaGraphExec_t ep_graph = nullptr;
    struct EpochKey {
        const void *X, *y, *idx;
        int B;
        float lr, wd;
        const void *bc, *losses;
        bool operator==(const EpochKey &o) const
        {
            return X == o.X && y == o.y && idx == o.idx && B == o.B && lr == o.lr && wd == o.wd && bc == o.bc &&
                   losses == o.losses;
        }
    } ep_key{};

    ~gn_mlp()
    {
        if (ep_graph) cudaGraphExecDestroy(ep_graph);
        ep_cursor.release();
        ep_bc.release();
        ep_losses.release();
        status.release();
        for (auto *a : {&params, &grads, &m, &v, &H2, &p, &part_w2, &part_w1, &part_head, &part_b1, &tmp_w1, &tmp_head})
            a->release();
        for (auto *a : {&W1t, &W2t, &W2b, &Xb, &H1, &dH2, &dH1, &XT, &H1T, &dH2T, &dH1T}) a->release();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Wait for the stream and report a device-side time-out.
void sync(gn_mlp *m, const char *what)
{
    cuda_check(cudaStreamSynchronize(m->stream), what);
    unsigned int st = 0;
    cuda_check(cudaMemcpy(&st, m->status.p, 4, cudaMemcpyDeviceToHost), "D2H status");
    if (st) {
        cudaMemset(m->status.p, 0, 4);
        fail(GN_ETIMEOUT, "a bounded device-side wait gave up (status %u)", st);
    }
}

void check_mlp(const gn_mlp *m)
{
    if (!m) fail(GN_EINVAL, "MLP handle is NULL");
}

void refresh(gn_mlp *m, cudaStream_t s)
{
    cuda_check(gn::mlp_launch_refresh(m->params.p + m->off_W1, m->in_dim, m->params.p + m->off_W2, m->W1t.p, m->W2t.p,
                                      m->W2b.p, s),
               "refresh");
}

// Rows of the batch per weight-gradient split: 256 when it divides Bp (32 splits,
// 128 CTAs for dW2 at the usual batch of 8192), else 128.
int wgrad_chunk(int Bp) { return Bp % 256 == 0 ? 256 : kChunk; }

// Forward pass of B rows (Bp padded) on stream s; with y, also the backward pass into
// m->grads and the mean loss into *loss (may be NULL).  With a device batch cursor the
// rows are idx[cursor B + b].
void run(gn_mlp *m, const float *X, const float *y, const int64_t *idx, int B, float *p_out, float *loss,
         const int64_t *cursor, cudaStream_t s)
{
    const int Bp = (B + kChunk - 1) / kChunk * kChunk;
    const float *P = m->params.p;
    cuda_check(gn::mlp_launch_cast(X, idx, cursor, B, m->in_dim, Bp, m->Xb.p, s), "cast");
    const bool train = y != nullptr;
    cuda_check(gn::mlp_launch_layer(0, m->Xb.p, Bp, KP, m->W1t.p, P + m->off_b1, nullptr, m->H1.p,
                                    train ? m->H1T.p : nullptr, nullptr, m->status.p, s),
               "layer 1");
    cuda_check(gn::mlp_launch_layer(1, m->H1.p, Bp, H, m->W2t.p, P + m->off_b2, nullptr, m->H2.p, nullptr, nullptr,
                                    m->status.p, s),
               "layer 2");
    cuda_check(gn::mlp_launch_head(m->H2.p, P + m->off_w3, P + m->off_b3, y, idx, cursor, B, Bp, kHeadRows, p_out, m->dH2.p,
                                   m->part_head.p, s),
               "head");
    if (!y) return;
    float *G = m->grads.p;
    // dH1 = (dH2 W2^T) [h1 > 0] and its column sums (db1)
    cuda_check(gn::mlp_launch_layer(2, m->dH2.p, Bp, H, m->W2b.p, nullptr, m->H1.p, m->dH1.p, m->dH1T.p, m->part_b1.p,
                                    m->status.p, s),
               "layer 2 backward");
    // weight gradients reduce over the batch: operands batch-contiguous, split over
    // `chunk` rows of the batch, partials summed in a fixed order
    cuda_check(gn::mlp_launch_transpose(m->dH2.p, Bp, H, m->dH2T.p, s), "transpose");
    cuda_check(gn::mlp_launch_transpose(m->Xb.p, Bp, KP, m->XT.p, s), "transpose");
    const int chunk = wgrad_chunk(Bp);
    cuda_check(gn::mlp_launch_wgrad(m->H1T.p, H, m->dH2T.p, H, Bp, chunk, false, m->part_w2.p, m->status.p, s), "dW2");
    cuda_check(gn::mlp_launch_wgrad(m->dH1T.p, H, m->XT.p, KP, Bp, chunk, true, m->part_w1.p, m->status.p, s), "dW1");
    const int nchunk = Bp / chunk, nhead = Bp / kHeadRows;
    cuda_check(gn::mlp_launch_sum(m->part_w2.p, nchunk, static_cast<int64_t>(H) * H, G + m->off_W2, s), "sum");
    cuda_check(gn::mlp_launch_sum(m->part_w1.p, nchunk, static_cast<int64_t>(KP) * H, m->tmp_w1.p, s), "sum");
    cuda_check(gn::mlp_launch_sum(m->part_b1.p, nhead, H, G + m->off_b1, s), "sum");
    cuda_check(gn::mlp_launch_sum(m->part_head.p, nhead, 2 * H + 2, m->tmp_head.p, s), "sum");
    cuda_check(cudaMemcpyAsync(G + m->off_W1, m->tmp_w1.p, sizeof(float) * m->in_dim * H, cudaMemcpyDeviceToDevice, s),
               "D2D");
    cuda_check(cudaMemcpyAsync(G + m->off_w3, m->tmp_head.p, sizeof(float) * H, cudaMemcpyDeviceToDevice, s), "D2D");
    cuda_check(cudaMemcpyAsync(G + m->off_b2, m->tmp_head.p + H, sizeof(float) * H, cudaMemcpyDeviceToDevice, s), "D2D");
    cuda_check(cudaMemcpyAsync(G + m->off_b3, m->tmp_head.p + 2 * H, sizeof(float), cudaMemcpyDeviceToDevice, s), "D2D");
    if (loss) {
        float sum = 0.0f;
        cuda_check(cudaMemcpyAsync(&sum, m->tmp_head.p + 2 * H + 1, sizeof(float), cudaMemcpyDeviceToHost, s), "D2H");
        sync(m, "MLP step");
        *loss = sum / static_cast<float>(B);
    }
}

}  // namespace

extern "C" {

gn_status gn_mlp_create(int32_t in_dim, int32_t max_batch, const float *params, int32_t device, void *cuda_stream,
                        gn_mlp **out)
{
    if (!out) {
        gnrt::set_error("out is NULL");
        return GN_EINVAL;
    }
    *out = nullptr;
    gn_mlp *m = nullptr;
    gn_status st = guarded([&] {
        if (in_dim < 1 || in_dim > KP) fail(GN_EINVAL, "in_dim must be in [1, %d]", KP);
        if (max_batch < 1 || max_batch > (1 << 24)) fail(GN_EINVAL, "max_batch out of range");
        if (!params) fail(GN_EINVAL, "params is NULL");
        m = new gn_mlp();
        m->device = device;
        DeviceGuard dg(device);
        if (cuda_stream) {
            m->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            cuda_check(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            m->own_stream = true;
        }
        m->in_dim = in_dim;
        m->max_bp = (max_batch + kChunk - 1) / kChunk * kChunk;
        m->off_W1 = 0;
        m->off_b1 = m->off_W1 + static_cast<int64_t>(in_dim) * H;
        m->off_W2 = m->off_b1 + H;
        m->off_b2 = m->off_W2 + static_cast<int64_t>(H) * H;
        m->off_w3 = m->off_b2 + H;
        m->off_b3 = m->off_w3 + H;
        m->n_params = m->off_b3 + 1;
        for (int64_t i = 0; i < m->n_params; ++i)
            if (!std::isfinite(params[i])) fail(GN_EINVAL, "parameter %lld is not finite", (long long)i);
        cuda_check(gn::mlp_prepare(), "MLP kernel setup");
        const size_t bp = m->max_bp;
        m->params.alloc(m->n_params, &m->bytes);
        m->grads.alloc(m->n_params, &m->bytes);
        m->m.alloc(m->n_params, &m->bytes);
        m->v.alloc(m->n_params, &m->bytes);
        m->W1t.alloc(static_cast<size_t>(H) * KP, &m->bytes);
        m->W2t.alloc(static_cast<size_t>(H) * H, &m->bytes);
        m->W2b.alloc(static_cast<size_t>(H) * H, &m->bytes);
        m->Xb.alloc(bp * KP, &m->bytes);
        m->H1.alloc(bp * H, &m->bytes);
        m->dH2.alloc(bp * H, &m->bytes);
        m->dH1.alloc(bp * H, &m->bytes);
        m->XT.alloc(bp * KP, &m->bytes);
        m->H1T.alloc(bp * H, &m->bytes);
        m->dH2T.alloc(bp * H, &m->bytes);
        m->dH1T.alloc(bp * H, &m->bytes);
        m->H2.alloc(bp * H, &m->bytes);
        m->p.alloc(bp, &m->bytes);
        m->part_w2.alloc(bp / kChunk * H * H, &m->bytes);
        m->part_w1.alloc(bp / kChunk * KP * H, &m->bytes);
        m->part_head.alloc(bp / kHeadRows * (2 * H + 2), &m->bytes);
        m->part_b1.alloc(bp / kHeadRows * H, &m->bytes);
        m->tmp_w1.alloc(static_cast<size_t>(KP) * H, &m->bytes);
        m->tmp_head.alloc(2 * H + 2, &m->bytes);
        m->status.alloc(1, &m->bytes);
        cuda_check(cudaMemset(m->status.p, 0, 4), "memset");
        cuda_check(cudaMemcpy(m->params.p, params, m->n_params * 4, cudaMemcpyHostToDevice), "H2D params");
        cuda_check(cudaMemset(m->grads.p, 0, m->n_params * 4), "memset");
        cuda_check(cudaMemset(m->m.p, 0, m->n_params * 4), "memset");
        cuda_check(cudaMemset(m->v.p, 0, m->n_params * 4), "memset");
        refresh(m, m->stream);
        cuda_check(cudaStreamSynchronize(m->stream), "create");
    });
    if (st != GN_OK) {
        delete m;
        return st;
    }
    *out = m;
    return GN_OK;
}

gn_status gn_mlp_destroy(gn_mlp *m)
{
    if (!m) return GN_OK;
    return guarded([&] {
        DeviceGuard dg(m->device);
        cudaStreamSynchronize(m->stream);
        delete m;
    });
}

gn_status gn_mlp_get_params(gn_mlp *m, float *params)
{
    return guarded([&] {
        check_mlp(m);
        if (!params) fail(GN_EINVAL, "params is NULL");
        DeviceGuard dg(m->device);
        sync(m, "MLP");
        cuda_check(cudaMemcpy(params, m->params.p, m->n_params * 4, cudaMemcpyDeviceToHost), "D2H params");
    });
}

gn_status gn_mlp_gradients(gn_mlp *m, const float *X, const float *y, const int64_t *idx, int32_t B, float *grads,
                           float *loss)
{
    return guarded([&] {
        check_mlp(m);
        if (B < 1 || B > m->max_bp || !X || !y || !grads) fail(GN_EINVAL, "bad batch (1 <= B <= max_batch)");
        DeviceGuard dg(m->device);
        float l = 0.0f;
        run(m, X, y, idx, B, m->p.p, &l, nullptr, m->stream);
        cuda_check(cudaMemcpy(grads, m->grads.p, m->n_params * 4, cudaMemcpyDeviceToHost), "D2H grads");
        if (loss) *loss = l;
    });
}

gn_status gn_mlp_train_step(gn_mlp *m, const float *X, const float *y, const int64_t *idx, int32_t B, float lr,
                            float weight_decay, float *loss)
{
    return guarded([&] {
        check_mlp(m);
        if (B < 1 || B > m->max_bp || !X || !y) fail(GN_EINVAL, "bad batch (1 <= B <= max_batch)");
        if (!(lr > 0.0f) || !(weight_decay >= 0.0f)) fail(GN_EINVAL, "bad learning rate or weight decay");
        DeviceGuard dg(m->device);
        run(m, X, y, idx, B, m->p.p, loss, nullptr, m->stream);
        // AdamW (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 masters
        m->adam_t += 1;
        const double t = static_cast<double>(m->adam_t);
        const float bc1 = static_cast<float>(1.0 - std::pow(0.9, t));
        const float bc2 = static_cast<float>(1.0 - std::pow(0.999, t));
        cuda_check(gn::mlp_launch_adamw(m->params.p, m->grads.p, m->m.p, m->v.p, m->n_params, lr, 0.9f, 0.999f, 1e-8f,
                                        weight_decay, bc1, bc2, nullptr, nullptr, m->stream),
                   "AdamW");
        refresh(m, m->stream);
    });
}

gn_status gn_mlp_train_epoch(gn_mlp *m, const float *X, const float *y, const int64_t *idx, int32_t n_batches,
                             int32_t B, float lr, float weight_decay, float *losses)
{
    return guarded([&] {
        check_mlp(m);
        if (B < 1 || B > m->max_bp || !X || !y || !idx || n_batches < 0)
            fail(GN_EINVAL, "bad batch (1 <= B <= max_batch, X, y, idx on the device)");
        if (!(lr > 0.0f) || !(weight_decay >= 0.0f)) fail(GN_EINVAL, "bad learning rate or weight decay");
        if (n_batches == 0) return;
        DeviceGuard dg(m->device);
        // AdamW bias corrections of steps adam_t + 1 .. adam_t + n_batches, as gn_mlp_train_step computes them
        std::vector<float> bc(2 * static_cast<size_t>(n_batches));
        for (int32_t j = 0; j < n_batches; ++j) {
            const double t = static_cast<double>(m->adam_t + 1 + j);
            bc[2 * j] = static_cast<float>(1.0 - std::pow(0.9, t));
            bc[2 * j + 1] = static_cast<float>(1.0 - std::pow(0.999, t));
        }
        if (m->ep_bc.n < bc.size() || m->ep_losses.n < static_cast<size_t>(n_batches) || !m->ep_cursor.p) {
            sync(m, "MLP");
            m->ep_bc.release();
            m->ep_losses.release();
            m->ep_bc.alloc(bc.size(), &m->bytes);
            m->ep_losses.alloc(n_batches, &m->bytes);
            if (!m->ep_cursor.p) m->ep_cursor.alloc(1, &m->bytes);
        }
        cuda_check(cudaMemcpyAsync(m->ep_bc.p, bc.data(), bc.size() * 4, cudaMemcpyHostToDevice, m->stream), "H2D");
        cuda_check(cudaMemsetAsync(m->ep_cursor.p, 0, 8, m->stream), "memset");
        const gn_mlp::EpochKey key{X, y, idx, B, lr, weight_decay, m->ep_bc.p, m->ep_losses.p};
        if (!m->ep_graph || !(key == m->ep_key)) {
            if (m->ep_graph) {
                cudaGraphExecDestroy(m->ep_graph);
                m->ep_graph = nullptr;
            }
            // one training step, the batch picked by the device cursor
            cudaStream_t cs;
            cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                try {
                    run(m, X, y, idx, B, m->p.p, nullptr, m->ep_cursor.p, cs);
                    cuda_check(gn::mlp_launch_adamw(m->params.p, m->grads.p, m->m.p, m->v.p, m->n_params, lr, 0.9f,
                                                    0.999f, 1e-8f, weight_decay, 1.0f, 1.0f, m->ep_bc.p,
                                                    m->ep_cursor.p, cs),
                               "AdamW");
                    refresh(m, cs);
                    cuda_check(gn::mlp_launch_epoch_tail(m->tmp_head.p + 2 * H + 1, B, m->ep_cursor.p, m->ep_losses.p,
                                                         cs),
                               "epoch tail");
                } catch (...) {
                    cudaStreamEndCapture(cs, &g);
                    if (g) cudaGraphDestroy(g);
                    cudaStreamDestroy(cs);
                    throw;
                }
                e = cudaStreamEndCapture(cs, &g);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&m->ep_graph, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            cuda_check(e, "graph capture of the training step");
            m->ep_key = key;
        }
        for (int32_t j = 0; j < n_batches; ++j) cuda_check(cudaGraphLaunch(m->ep_graph, m->stream), "cudaGraphLaunch");
        m->adam_t += n_batches;
        if (losses) {
            cuda_check(cudaMemcpyAsync(losses, m->ep_losses.p, static_cast<size_t>(n_batches) * 4,
                                       cudaMemcpyDeviceToHost, m->stream),
                       "D2H losses");
            sync(m, "MLP epoch");
        }
    });
}

gn_status gn_mlp_infer(gn_mlp *m, const float *X, int64_t B, float *p)
{
    return guarded([&] {
        check_mlp(m);
        if (B < 0 || (B > 0 && (!X || !p))) fail(GN_EINVAL, "bad batch");
        DeviceGuard dg(m->device);
        for (int64_t b0 = 0; b0 < B; b0 += m->max_bp) {
            const int nb = static_cast<int>(std::min<int64_t>(m->max_bp, B - b0));
            run(m, X + b0 * m->in_dim, nullptr, nullptr, nb, p + b0, nullptr, nullptr, m->stream);
        }
    });
}

gn_status gn_mlp_synchronize(gn_mlp *m)
{
    return guarded([&] {
        check_mlp(m);
        DeviceGuard dg(m->device);
        sync(m, "MLP");
    });
}

}  // extern "C"
