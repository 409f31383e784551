// Host runtime of the learned estimator (gn_mlp_* in include/geonet.h): an MLP
// in -> 256 -> 256 -> 1 trained with the project's own forward, backward and
// AdamW kernels (k_mlp.cu) on device-resident batches.
//
// Parameters, gradients and Adam moments are packed FP32 buffers in one layout,
// [W1 (in x 256) | b1 | W2 (256 x 256) | b2 | w3 | b3]; the BF16 weight images the
// tile kernel streams are rewritten by every AdamW step.  A training step is three
// launches: the tile kernel (forward, loss, dH2, dH1), the weight-gradient GEMMs and
// the update (fixed-order sums, AdamW, images; in a replayed epoch also the loss of
// the step and the batch cursor).  A replayed epoch runs graphs of 16 steps, the
// launches chained by programmatic dependent launch across the steps.
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
constexpr int kTileRows = 128;  // batch padding granularity (rows of one tile)
constexpr int kEpochGraphSteps = 16;  // training steps per replayed graph of an epoch
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
    DevArray<uint8_t> wimg, xt_img, h1t_img, dh2t_img, dh1t_img;
    DevArray<float> p, part_w2, part_w1, part_head, part_b1, loss_sum;
    DevArray<unsigned int> status;  // kStatusTimeout when a kernel's bounded wait gave up
    // replayed training epochs: batch cursor, bias-correction table, per-step losses
    DevArray<int64_t> ep_cursor;
    DevArray<unsigned int> ep_ticket;  // the update kernel's count of finished CTAs (zero between steps)
    DevArray<float> ep_bc, ep_losses;
    // kEpochGraphSteps steps chained in one graph (programmatic dependent launch across
    // the steps too), and one step for the remainder
    cudaGraphExec_t ep_graph = nullptr, ep_graph1 = nullptr;
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

    gn::MlpBuffers buffers() const
    {
        gn::MlpBuffers b{};
        b.in_dim = in_dim;
        b.n_params = n_params;
        b.off_W1 = off_W1;
        b.off_b1 = off_b1;
        b.off_W2 = off_W2;
        b.off_b2 = off_b2;
        b.off_w3 = off_w3;
        b.off_b3 = off_b3;
        b.params = params.p;
        b.grads = grads.p;
        b.m = m.p;
        b.v = v.p;
        b.wimg = wimg.p;
        b.xt_img = xt_img.p;
        b.h1t_img = h1t_img.p;
        b.dh2t_img = dh2t_img.p;
        b.dh1t_img = dh1t_img.p;
        b.part_w2 = part_w2.p;
        b.part_w1 = part_w1.p;
        b.part_head = part_head.p;
        b.part_b1 = part_b1.p;
        b.loss_sum = loss_sum.p;
        b.status = status.p;
        return b;
    }

    ~gn_mlp()
    {
        if (ep_graph) cudaGraphExecDestroy(ep_graph);
        if (ep_graph1) cudaGraphExecDestroy(ep_graph1);
        ep_cursor.release();
        ep_ticket.release();
        ep_bc.release();
        ep_losses.release();
        status.release();
        for (auto *a : {&params, &grads, &m, &v, &p, &part_w2, &part_w1, &part_head, &part_b1, &loss_sum}) a->release();
        for (auto *a : {&wimg, &xt_img, &h1t_img, &dh2t_img, &dh1t_img}) a->release();
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

int padded(int B) { return (B + kTileRows - 1) / kTileRows * kTileRows; }

// Forward pass of B rows on stream s; with y, also the backward pass into m->grads
// (and the loss sum on the device), then with `adamw` the AdamW step.  With a device
// batch cursor the rows are idx[cursor B + b] and the bias corrections come from
// bc_table.
void run(gn_mlp *m, const float *X, const float *y, const int64_t *idx, int B, float *p_out, int64_t *cursor,
         bool adamw, float lr, float wd, float bc1, float bc2, const float *bc_table, cudaStream_t s,
         float *losses = nullptr)
{
    const int Bp = padded(B);
    const gn::MlpBuffers b = m->buffers();
    cuda_check(gn::mlp_launch_tile(b, X, idx, cursor, y, B, Bp, p_out, s), "MLP tile kernel");
    if (!y) return;
    cuda_check(gn::mlp_launch_wgrad(b, Bp, s), "MLP weight gradients");
    cuda_check(gn::mlp_launch_update(b, Bp, adamw, lr, wd, bc1, bc2, bc_table, cursor, losses,
                                     losses ? m->ep_ticket.p : nullptr, B, s),
               "MLP update");
}

float read_loss(gn_mlp *m, int B)
{
    float sum = 0.0f;
    cuda_check(cudaMemcpyAsync(&sum, m->loss_sum.p, sizeof(float), cudaMemcpyDeviceToHost, m->stream), "D2H");
    sync(m, "MLP step");
    return sum / static_cast<float>(B);
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
        if (in_dim < 1 || in_dim > gn::kMlpInPad) fail(GN_EINVAL, "in_dim must be in [1, %d]", gn::kMlpInPad);
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
        m->max_bp = padded(max_batch);
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
        const int bp = m->max_bp;
        int cps = 0;
        const int splits = gn::mlp_wgrad_splits(bp, &cps);
        m->params.alloc(m->n_params, &m->bytes);
        m->grads.alloc(m->n_params, &m->bytes);
        m->m.alloc(m->n_params, &m->bytes);
        m->v.alloc(m->n_params, &m->bytes);
        m->wimg.alloc(gn::mlp_wimg_bytes(), &m->bytes);
        m->xt_img.alloc(gn::mlp_xt_bytes(bp), &m->bytes);
        m->h1t_img.alloc(gn::mlp_ht_bytes(bp), &m->bytes);
        m->dh2t_img.alloc(gn::mlp_ht_bytes(bp), &m->bytes);
        m->dh1t_img.alloc(gn::mlp_ht_bytes(bp), &m->bytes);
        m->p.alloc(bp, &m->bytes);
        m->part_w2.alloc(static_cast<size_t>(splits) * H * H, &m->bytes);
        m->part_w1.alloc(static_cast<size_t>(splits) * H * gn::kMlpInPad, &m->bytes);
        m->part_head.alloc(static_cast<size_t>(bp / kTileRows) * (2 * H + 2), &m->bytes);
        m->part_b1.alloc(static_cast<size_t>(bp / kTileRows) * H, &m->bytes);
        m->loss_sum.alloc(1, &m->bytes);
        m->status.alloc(1, &m->bytes);
        cuda_check(cudaMemset(m->status.p, 0, 4), "memset");
        cuda_check(cudaMemset(m->wimg.p, 0, gn::mlp_wimg_bytes()), "memset");
        cuda_check(cudaMemcpy(m->params.p, params, m->n_params * 4, cudaMemcpyHostToDevice), "H2D params");
        cuda_check(cudaMemset(m->grads.p, 0, m->n_params * 4), "memset");
        cuda_check(cudaMemset(m->m.p, 0, m->n_params * 4), "memset");
        cuda_check(cudaMemset(m->v.p, 0, m->n_params * 4), "memset");
        cuda_check(gn::mlp_launch_refresh(m->buffers(), m->stream), "weight images");
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
        run(m, X, y, idx, B, m->p.p, nullptr, false, 0.0f, 0.0f, 1.0f, 1.0f, nullptr, m->stream);
        const float l = read_loss(m, B);
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
        // AdamW (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 masters
        m->adam_t += 1;
        const double t = static_cast<double>(m->adam_t);
        const float bc1 = static_cast<float>(1.0 - std::pow(0.9, t));
        const float bc2 = static_cast<float>(1.0 - std::pow(0.999, t));
        run(m, X, y, idx, B, m->p.p, nullptr, true, lr, weight_decay, bc1, bc2, nullptr, m->stream);
        if (loss) *loss = read_loss(m, B);
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
            if (!m->ep_ticket.p) {
                m->ep_ticket.alloc(1, &m->bytes);
                cuda_check(cudaMemset(m->ep_ticket.p, 0, 4), "memset");
            }
        }
        cuda_check(cudaMemcpyAsync(m->ep_bc.p, bc.data(), bc.size() * 4, cudaMemcpyHostToDevice, m->stream), "H2D");
        cuda_check(cudaMemsetAsync(m->ep_cursor.p, 0, 8, m->stream), "memset");
        const gn_mlp::EpochKey key{X, y, idx, B, lr, weight_decay, m->ep_bc.p, m->ep_losses.p};
        if (!(key == m->ep_key)) {
            for (cudaGraphExec_t *ge : {&m->ep_graph, &m->ep_graph1})
                if (*ge) {
                    cudaGraphExecDestroy(*ge);
                    *ge = nullptr;
                }
        }
        // `steps` training steps, each taking the batch the device cursor points at
        auto capture = [&](int steps) {
            cudaStream_t cs;
            cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                try {
                    for (int j = 0; j < steps; ++j)
                        run(m, X, y, idx, B, m->p.p, m->ep_cursor.p, true, lr, weight_decay, 1.0f, 1.0f, m->ep_bc.p,
                            cs, m->ep_losses.p);
                } catch (...) {
                    cudaStreamEndCapture(cs, &g);
                    if (g) cudaGraphDestroy(g);
                    cudaStreamDestroy(cs);
                    throw;
                }
                e = cudaStreamEndCapture(cs, &g);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            cuda_check(e, "graph capture of the training steps");
            return ge;
        };
        const int32_t full = n_batches / kEpochGraphSteps, rest = n_batches % kEpochGraphSteps;
        if (full && !m->ep_graph) m->ep_graph = capture(kEpochGraphSteps);
        if (rest && !m->ep_graph1) m->ep_graph1 = capture(1);
        m->ep_key = key;
        for (int32_t j = 0; j < full; ++j) cuda_check(cudaGraphLaunch(m->ep_graph, m->stream), "cudaGraphLaunch");
        for (int32_t j = 0; j < rest; ++j) cuda_check(cudaGraphLaunch(m->ep_graph1, m->stream), "cudaGraphLaunch");
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
            run(m, X + b0 * m->in_dim, nullptr, nullptr, nb, p + b0, nullptr, false, 0.0f, 0.0f, 1.0f, 1.0f, nullptr,
                m->stream);
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
