// proposal.cu -- C ABI of the learned proposal network (nn.cu kernels).
//
// Host code validates arguments, owns the network's device memory and
// launches kernels; all arithmetic runs on the device.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pfreg.h"
#include "kernels.h"
#include "nn.h"

namespace pfreg {
int set_error(int code, const char *msg);
cudaError_t nn_error_flag(unsigned int *out, bool clear);
cudaError_t nn_wait_selftest(cudaStream_t s);
cudaError_t nn_gemm(const uint16_t *A, const uint16_t *B, float *C, int M, int K, cudaStream_t s);
cudaError_t nn_conv_fwd(const uint16_t *X, int batch, int D, int Cin, const uint16_t *W, const float *bias,
                        uint16_t *Y, cudaStream_t s);
cudaError_t nn_conv_dgrad(const uint16_t *dY, int batch, int D, const uint16_t *Wt, const uint16_t *act,
                          uint16_t *dX, cudaStream_t s);
cudaError_t nn_conv_wgrad(const uint16_t *X, int batch, int D, int Cin, const uint16_t *dY, float *dW,
                          cudaStream_t s);
cudaError_t nn_transpose_w(const uint16_t *W, int Cin, uint16_t *Wt, cudaStream_t s);

// the network's passes (nn.cu)
cudaError_t net_forward(const NetPtrs &n, int B, cudaStream_t s);
cudaError_t net_backward(const NetPtrs &n, int B, cudaStream_t s);
cudaError_t net_adam(const NetPtrs &n, float lr, cudaStream_t s);
cudaError_t net_init(const NetPtrs &n, uint64_t seed, cudaStream_t s);
cudaError_t net_refresh_bf16(const NetPtrs &n, cudaStream_t s);
cudaError_t net_synth(const NetPtrs &n, int B, uint64_t seed, int step, float rot_lim, float trans_lim,
                      const int dims[3], bool step_from_counter, cudaStream_t s);
size_t net_sample_bytes();
cudaError_t net_downsample(const NetPtrs &n, const uint8_t *vol, const int dims[3], const float origin[3],
                           const float spacing[3], const float box_o[3], const float box_h[3], int channel,
                           cudaStream_t s);
}  // namespace pfreg

using namespace pfreg;

namespace {

int cuda_fail(cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return set_error(e == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, buf);
}

#define CUP(call)                                             \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// After a synchronising call: a tensor-core kernel whose bounded mbarrier
// wait ran out left its tile unwritten.  Report that as PF_ETIMEOUT (and
// clear the flag, so that the next call starts clean).
int check_waits() {
    unsigned int f = 0;
    CUP(nn_error_flag(&f, false));
    if (!f) return PF_OK;
    CUP(nn_error_flag(&f, true));
    return set_error(PF_ETIMEOUT, "a tensor-core kernel's bounded wait ran out; its output tile was not written");
}

// Rows of a conv's implicit GEMM must stay within int32, and D must halve.
int check_conv(int batch, int D, int Cin) {
    if (batch < 1 || D < 2 || (D & 1) || D > 512) return set_error(PF_EINVAL, "conv: batch >= 1, D even in [2, 512]");
    if (!(Cin == 2 || Cin == 8 || Cin == 16 || Cin == 32 || Cin == 64 || Cin == 128 || Cin == 256))
        return set_error(PF_EINVAL, "conv: Cin must be 2, 8, 16, 32, 64, 128 or 256");
    if ((long long)batch * D * D * D >= (1ll << 31) / 64) return set_error(PF_EINVAL, "conv: volume too large");
    return PF_OK;
}

}  // namespace

extern "C" {

int pf_nn_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int32_t M, int32_t K, void *stream) {
    if (!A || !B || !C) return set_error(PF_EINVAL, "gemm: NULL pointer");
    if (M < 1 || K < 8 || K % 8 || (long long)M * K >= (1ll << 31)) return set_error(PF_EINVAL, "gemm: M >= 1, K >= 8, K % 8 == 0");
    CUP(nn_gemm(A, B, C, M, K, static_cast<cudaStream_t>(stream)));
    return PF_OK;
}

int pf_nn_conv3d_forward(const uint16_t *x, int32_t batch, int32_t D, int32_t Cin, const uint16_t *w,
                         const float *bias, uint16_t *y, void *stream) {
    if (!x || !w || !bias || !y) return set_error(PF_EINVAL, "conv forward: NULL pointer");
    if (int r = check_conv(batch, D, Cin)) return r;
    CUP(nn_conv_fwd(x, batch, D, Cin, w, bias, y, static_cast<cudaStream_t>(stream)));
    return PF_OK;
}

int pf_nn_conv3d_backward_data(const uint16_t *dy, int32_t batch, int32_t D, const uint16_t *w_t,
                               const uint16_t *act, uint16_t *dx, void *stream) {
    if (!dy || !w_t || !dx) return set_error(PF_EINVAL, "conv backward data: NULL pointer");
    if (int r = check_conv(batch, D, 32)) return r;
    CUP(nn_conv_dgrad(dy, batch, D, w_t, act, dx, static_cast<cudaStream_t>(stream)));
    return PF_OK;
}

int pf_nn_conv3d_backward_weights(const uint16_t *x, int32_t batch, int32_t D, int32_t Cin, const uint16_t *dy,
                                  float *dw, void *stream) {
    if (!x || !dy || !dw) return set_error(PF_EINVAL, "conv backward weights: NULL pointer");
    if (int r = check_conv(batch, D, Cin)) return r;
    CUP(nn_conv_wgrad(x, batch, D, Cin, dy, dw, static_cast<cudaStream_t>(stream)));
    return PF_OK;
}

int pf_nn_wait_selftest(void *stream) {
    CUP(nn_wait_selftest(static_cast<cudaStream_t>(stream)));
    return PF_OK;
}

int pf_nn_status(int32_t clear, int32_t *gave_up) {
    if (!gave_up) return set_error(PF_EINVAL, "status: NULL pointer");
    unsigned int f = 0;
    CUP(nn_error_flag(&f, clear != 0));
    *gave_up = (int32_t)f;
    return PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The proposal network object.
// ---------------------------------------------------------------------------
struct pf_proposal {
    cudaStream_t stream = nullptr;
    NetPtrs n{};
    std::vector<void *> allocs;
    float rot_lim = 0.0f, trans_lim = 0.0f;   // units of the outputs (set by training)
    float *loss_log = nullptr;
    int loss_cap = 0;
    cudaGraphExec_t train_exec = nullptr;
    int train_batch = 0;
    float train_lr = 0.0f;
    uint64_t train_seed = 0;
    int train_dims[3] = {0, 0, 0};
    float train_rl = 0.0f, train_tl = 0.0f;

    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = dev_malloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 1);
        if (e == cudaSuccess) {
            allocs.push_back(q);
            *p = static_cast<T *>(q);
        }
        return e;
    }
    ~pf_proposal() {
        if (train_exec) cudaGraphExecDestroy(train_exec);
        if (loss_log) cudaFree(loss_log);
        for (void *p : allocs) cudaFree(p);
    }
};

namespace {

// One training step: synthetic batch, forward, backward, Adam.
cudaError_t train_step(pf_proposal *p, cudaStream_t s) {
    cudaError_t e = net_synth(p->n, p->train_batch, p->train_seed, 0, p->train_rl, p->train_tl, p->train_dims,
                              true, s);
    if (e == cudaSuccess) e = net_forward(p->n, p->train_batch, s);
    if (e == cudaSuccess) e = net_backward(p->n, p->train_batch, s);
    if (e == cudaSuccess) e = net_adam(p->n, p->train_lr, s);
    return e;
}

int copy_volume_to_device(const pf_volume *v, const uint8_t **dev, uint8_t **owned, cudaStream_t s) {
    const size_t n = (size_t)v->dims[0] * v->dims[1] * v->dims[2];
    *owned = nullptr;
    if (v->is_device) {
        *dev = static_cast<const uint8_t *>(v->data);
        return PF_OK;
    }
    CUP(dev_malloc_async(owned, n, s));
    CUP(cudaMemcpyAsync(*owned, v->data, n, cudaMemcpyHostToDevice, s));
    *dev = *owned;
    return PF_OK;
}

bool volume_ok(const pf_volume *v) {
    if (!v || !v->data) return false;
    for (int d = 0; d < 3; ++d) {
        if (v->dims[d] < 2 || v->dims[d] > 2048) return false;
        if (!std::isfinite(v->origin[d]) || !(v->spacing[d] > 0.0f && v->spacing[d] <= 1e6f)) return false;
    }
    return true;
}

}  // namespace

extern "C" {

int pf_proposal_create(pf_proposal **out, int32_t max_batch, uint64_t seed, void *stream) {
    if (!out) return set_error(PF_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > 256) return set_error(PF_EINVAL, "max_batch outside [1, 256]");
    pf_proposal *p = new (std::nothrow) pf_proposal();
    if (!p) return set_error(PF_ENOMEM, "host allocation failed");
    p->stream = static_cast<cudaStream_t>(stream);
    NetPtrs &n = p->n;
    n.max_batch = max_batch;
    const long long P = n.L.total;
    const size_t B = (size_t)max_batch;
    auto bail = [&](cudaError_t e, const char *what) {
        delete p;
        return cuda_fail(e, what);
    };
#define PA(ptr, count)                                   \
    do {                                                 \
        cudaError_t e_ = p->alloc(&(ptr), (count));      \
        if (e_ != cudaSuccess) return bail(e_, #ptr);    \
    } while (0)
    PA(n.theta, P);
    PA(n.grad, P);
    PA(n.m, P);
    PA(n.v, P);
    for (int l = 0; l < 4; ++l) {
        PA(n.wbf[l], 32 * 64 * (size_t)net_cin(l));
        n.wt[l] = nullptr;
        if (l > 0) PA(n.wt[l], 32 * 64 * 32);
        const size_t e = (size_t)(net_din(l) / 2);
        PA(n.a[l], B * e * e * e * 32);
        PA(n.d[l], B * e * e * e * 32);
    }
    PA(n.x, B * kNetG * kNetG * kNetG * 2);
    PA(n.h, B * kNetHidden);
    PA(n.dh, B * kNetHidden);
    PA(n.out, B * kNetOut);
    PA(n.dout, B * kNetOut);
    PA(n.y, B * 6);
    PA(n.step, 1);
    uint8_t *smp = nullptr;
    PA(smp, B * net_sample_bytes());
    n.samples = smp;
    float *loss0 = nullptr;
    PA(loss0, 1);
    n.loss = loss0;
#undef PA
    cudaError_t e = net_init(n, seed, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return bail(e, "network initialisation");
    *out = p;
    return PF_OK;
}

int pf_proposal_destroy(pf_proposal *p) {
    delete p;
    return PF_OK;
}

int pf_proposal_train(pf_proposal *p, int32_t n_steps, int32_t batch, float lr, uint64_t data_seed,
                      const int32_t vol_dims[3], float rot_limit, float trans_limit, float *loss_out) {
    if (!p || !vol_dims) return set_error(PF_EINVAL, "NULL argument");
    if (n_steps < 0 || n_steps > (1 << 24)) return set_error(PF_EINVAL, "n_steps outside [0, 2^24]");
    if (batch < 1 || batch > p->n.max_batch) return set_error(PF_EINVAL, "batch outside [1, max_batch]");
    if (!(lr > 0.0f && lr < 1.0f)) return set_error(PF_EINVAL, "lr outside (0, 1)");
    if (!(rot_limit > 0.0f && rot_limit <= 1.5707964f) || !(trans_limit > 0.0f && trans_limit <= 2048.0f))
        return set_error(PF_EINVAL, "limits outside (0, pi/2] / (0, 2048]");
    for (int d = 0; d < 3; ++d)
        if (vol_dims[d] < kNetG || vol_dims[d] > 1024) return set_error(PF_EINVAL, "vol_dims outside [64, 1024]");
    if (p->rot_lim != 0.0f && (p->rot_lim != rot_limit || p->trans_lim != trans_limit))
        return set_error(PF_EINVAL, "limits differ from the ones the network was trained with");
    cudaStream_t s = p->stream;
    if (n_steps == 0) return PF_OK;
    // the per-step loss log, indexed by the step counter
    int32_t step0 = 0;
    CUP(cudaMemcpyAsync(&step0, p->n.step, sizeof step0, cudaMemcpyDeviceToHost, s));
    CUP(cudaStreamSynchronize(s));
    const int need = step0 + n_steps;
    if (need > p->loss_cap) {
        float *nl = nullptr;
        CUP(dev_malloc(&nl, sizeof(float) * (size_t)need));
        CUP(cudaMemsetAsync(nl, 0, sizeof(float) * (size_t)need, s));
        if (p->loss_log && step0 > 0) CUP(cudaMemcpyAsync(nl, p->loss_log, sizeof(float) * step0, cudaMemcpyDeviceToDevice, s));
        CUP(cudaStreamSynchronize(s));
        if (p->loss_log) cudaFree(p->loss_log);
        p->loss_log = nl;
        p->loss_cap = need;
        if (p->train_exec) cudaGraphExecDestroy(p->train_exec);   // captured with the old log
        p->train_exec = nullptr;
    }
    p->n.loss = p->loss_log;
    const bool same = p->train_exec && p->train_batch == batch && p->train_lr == lr && p->train_seed == data_seed &&
                      p->train_rl == rot_limit && p->train_tl == trans_limit && p->train_dims[0] == vol_dims[0] &&
                      p->train_dims[1] == vol_dims[1] && p->train_dims[2] == vol_dims[2];
    if (!same) {
        if (p->train_exec) cudaGraphExecDestroy(p->train_exec);
        p->train_exec = nullptr;
        p->train_batch = batch;
        p->train_lr = lr;
        p->train_seed = data_seed;
        p->train_rl = rot_limit;
        p->train_tl = trans_limit;
        for (int d = 0; d < 3; ++d) p->train_dims[d] = vol_dims[d];
        // one training step as a CUDA graph (the step index lives on the device)
        cudaStream_t cap = nullptr;
        CUP(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = train_step(p, cap);
            e = cudaStreamEndCapture(cap, &graph);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->train_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_fail(e, "training graph");
    }
    p->rot_lim = rot_limit;
    p->trans_lim = trans_limit;
    for (int32_t i = 0; i < n_steps; ++i) {
        CUP(cudaGraphLaunch(p->train_exec, s));
        count_launches(40);
    }
    if (loss_out) {
        CUP(cudaMemcpyAsync(loss_out, p->loss_log + step0, sizeof(float) * (size_t)n_steps, cudaMemcpyDeviceToHost, s));
        CUP(cudaStreamSynchronize(s));
        return check_waits();
    }
    return PF_OK;
}

int pf_proposal_predict(pf_proposal *p, const pf_volume *src, const pf_volume *tgt, float mean_out[6],
                        float std_out[6]) {
    if (!p || !mean_out || !std_out) return set_error(PF_EINVAL, "NULL argument");
    if (!volume_ok(src) || !volume_ok(tgt)) return set_error(PF_EINVAL, "bad src / tgt volume");
    if (p->rot_lim == 0.0f) return set_error(PF_ESTATE, "the network has not been trained");
    cudaStream_t s = p->stream;
    const uint8_t *ds = nullptr, *dt = nullptr;
    uint8_t *os = nullptr, *ot = nullptr;
    int rc = copy_volume_to_device(src, &ds, &os, s);
    if (!rc) rc = copy_volume_to_device(tgt, &dt, &ot, s);
    float box_h[3];
    for (int d = 0; d < 3; ++d) box_h[d] = src->spacing[d] * (float)src->dims[d] / (float)kNetG;
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = net_downsample(p->n, ds, src->dims, src->origin, src->spacing, src->origin, box_h, 0, s);
        if (e == cudaSuccess) e = net_downsample(p->n, dt, tgt->dims, tgt->origin, tgt->spacing, src->origin, box_h, 1, s);
        if (e == cudaSuccess) e = net_forward(p->n, 1, s);
    }
    float out[kNetOut];
    if (!rc && e == cudaSuccess) e = cudaMemcpyAsync(out, p->n.out, sizeof out, cudaMemcpyDeviceToHost, s);
    if (os) cudaFreeAsync(os, s);
    if (ot) cudaFreeAsync(ot, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (rc) return rc;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "proposal forward");
    if ((rc = check_waits())) return rc;
    for (int d = 0; d < 6; ++d) {
        const float unit = d < 3 ? p->rot_lim : p->trans_lim;
        mean_out[d] = out[d] * unit;
        std_out[d] = expf(0.5f * fminf(fmaxf(out[6 + d], -30.0f), 30.0f)) * unit;
    }
    return PF_OK;
}

int pf_proposal_params(pf_proposal *p, float *theta_out, float *grad_out, const float *theta_in, int64_t *n_params) {
    if (!p || !n_params) return set_error(PF_EINVAL, "NULL argument");
    const long long P = p->n.L.total;
    *n_params = P;
    cudaStream_t s = p->stream;
    if (theta_in) {
        CUP(cudaMemcpyAsync(p->n.theta, theta_in, sizeof(float) * P, cudaMemcpyHostToDevice, s));
        CUP(net_refresh_bf16(p->n, s));
    }
    if (theta_out) CUP(cudaMemcpyAsync(theta_out, p->n.theta, sizeof(float) * P, cudaMemcpyDeviceToHost, s));
    if (grad_out) CUP(cudaMemcpyAsync(grad_out, p->n.grad, sizeof(float) * P, cudaMemcpyDeviceToHost, s));
    CUP(cudaStreamSynchronize(s));
    return PF_OK;
}

int pf_proposal_forward(pf_proposal *p, const uint16_t *x, int32_t batch, float *out, float *hidden) {
    if (!p || !x || !out) return set_error(PF_EINVAL, "NULL argument");
    if (batch < 1 || batch > p->n.max_batch) return set_error(PF_EINVAL, "batch outside [1, max_batch]");
    cudaStream_t s = p->stream;
    CUP(cudaMemcpyAsync(p->n.x, x, sizeof(uint16_t) * (size_t)batch * kNetG * kNetG * kNetG * 2,
                        cudaMemcpyDeviceToDevice, s));
    CUP(net_forward(p->n, batch, s));
    CUP(cudaMemcpyAsync(out, p->n.out, sizeof(float) * (size_t)batch * kNetOut, cudaMemcpyDeviceToDevice, s));
    if (hidden) CUP(cudaMemcpyAsync(hidden, p->n.h, sizeof(float) * (size_t)batch * kNetHidden, cudaMemcpyDeviceToDevice, s));
    return PF_OK;
}

int pf_proposal_backward(pf_proposal *p, const float *y, int32_t batch, float *loss_out) {
    if (!p || !y) return set_error(PF_EINVAL, "NULL argument");
    if (batch < 1 || batch > p->n.max_batch) return set_error(PF_EINVAL, "batch outside [1, max_batch]");
    cudaStream_t s = p->stream;
    CUP(cudaMemcpyAsync(p->n.y, y, sizeof(float) * (size_t)batch * 6, cudaMemcpyDeviceToDevice, s));
    // the loss of this call goes to a scratch slot: the log entry of the current step
    float *scratch = nullptr;
    CUP(dev_malloc_async(&scratch, sizeof(float), s));
    CUP(cudaMemsetAsync(scratch, 0, sizeof(float), s));
    NetPtrs n = p->n;
    n.loss = scratch;
    int *zero = nullptr;
    CUP(dev_malloc_async(&zero, sizeof(int), s));
    CUP(cudaMemsetAsync(zero, 0, sizeof(int), s));
    n.step = zero;
    cudaError_t e = net_backward(n, batch, s);
    float l = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, scratch, sizeof l, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(scratch, s);
    cudaFreeAsync(zero, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "proposal backward");
    if (loss_out) *loss_out = l;
    return check_waits();
}

int pf_proposal_tensor(pf_proposal *p, int32_t which, int32_t batch, void *host_out) {
    if (!p || !host_out) return set_error(PF_EINVAL, "NULL argument");
    if (batch < 1 || batch > p->n.max_batch) return set_error(PF_EINVAL, "batch outside [1, max_batch]");
    const void *src = nullptr;
    size_t bytes = 0;
    if (which >= 0 && which < 8) {
        const int l = which & 3;
        const long long D = kNetG >> (l + 1);
        src = which < 4 ? (const void *)p->n.a[l] : (const void *)p->n.d[l];
        bytes = sizeof(uint16_t) * (size_t)batch * D * D * D * 32;
    } else if (which == 8 || which == 10) {
        src = which == 8 ? p->n.h : p->n.dh;
        bytes = sizeof(float) * (size_t)batch * kNetHidden;
    } else if (which == 9 || which == 11) {
        src = which == 9 ? p->n.out : p->n.dout;
        bytes = sizeof(float) * (size_t)batch * kNetOut;
    } else {
        return set_error(PF_EINVAL, "which outside [0, 11]");
    }
    CUP(cudaMemcpyAsync(host_out, src, bytes, cudaMemcpyDeviceToHost, p->stream));
    CUP(cudaStreamSynchronize(p->stream));
    return PF_OK;
}

int pf_proposal_synth(pf_proposal *p, int32_t batch, uint64_t seed, int32_t step, const int32_t vol_dims[3],
                      float rot_limit, float trans_limit, uint16_t *x_out, float *y_out) {
    if (!p || !vol_dims || !x_out || !y_out) return set_error(PF_EINVAL, "NULL argument");
    if (batch < 1 || batch > p->n.max_batch) return set_error(PF_EINVAL, "batch outside [1, max_batch]");
    for (int d = 0; d < 3; ++d)
        if (vol_dims[d] < kNetG || vol_dims[d] > 1024) return set_error(PF_EINVAL, "vol_dims outside [64, 1024]");
    if (!(rot_limit > 0.0f) || !(trans_limit > 0.0f)) return set_error(PF_EINVAL, "limits must be > 0");
    cudaStream_t s = p->stream;
    CUP(net_synth(p->n, batch, seed, step, rot_limit, trans_limit, vol_dims, false, s));
    CUP(cudaMemcpyAsync(x_out, p->n.x, sizeof(uint16_t) * (size_t)batch * kNetG * kNetG * kNetG * 2,
                        cudaMemcpyDeviceToDevice, s));
    CUP(cudaMemcpyAsync(y_out, p->n.y, sizeof(float) * (size_t)batch * 6, cudaMemcpyDeviceToDevice, s));
    return PF_OK;
}

int pf_proposal_input(pf_proposal *p, const pf_volume *src, const pf_volume *tgt, uint16_t *x_out) {
    if (!p || !x_out) return set_error(PF_EINVAL, "NULL argument");
    if (!volume_ok(src) || !volume_ok(tgt)) return set_error(PF_EINVAL, "bad src / tgt volume");
    cudaStream_t s = p->stream;
    const uint8_t *ds = nullptr, *dt = nullptr;
    uint8_t *os = nullptr, *ot = nullptr;
    int rc = copy_volume_to_device(src, &ds, &os, s);
    if (!rc) rc = copy_volume_to_device(tgt, &dt, &ot, s);
    float box_h[3];
    for (int d = 0; d < 3; ++d) box_h[d] = src->spacing[d] * (float)src->dims[d] / (float)kNetG;
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = net_downsample(p->n, ds, src->dims, src->origin, src->spacing, src->origin, box_h, 0, s);
        if (e == cudaSuccess) e = net_downsample(p->n, dt, tgt->dims, tgt->origin, tgt->spacing, src->origin, box_h, 1, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x_out, p->n.x, sizeof(uint16_t) * kNetG * kNetG * kNetG * 2, cudaMemcpyDeviceToDevice, s);
    }
    if (os) cudaFreeAsync(os, s);
    if (ot) cudaFreeAsync(ot, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (rc) return rc;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return cuda_fail(e, "proposal input");
    return PF_OK;
}

}  // extern "C"
