// nn.h -- the learned proposal network's parameter layout and device buffers
// (shared by the kernels in nn.cu and the C ABI in proposal.cu).
//
// Architecture: input [B][64^3][2] (source and target box-averaged onto one
// 64^3 grid over the source's box), four convolutions of kernel 4^3, stride
// 2, padding 1 and 32 channels with ReLU (64^3 -> 32^3 -> 16^3 -> 8^3 ->
// 4^3), a fully connected layer 2048 -> 128 with ReLU and a linear layer
// 128 -> 12 giving the pose mean (6) and log-variance (6), both in units of
// the training limits.  464,652 parameters.
#pragma once
#include <cstdint>

namespace pfreg {

constexpr int kNetG = 64;
constexpr int kNetHidden = 128;
constexpr int kNetOut = 12;
constexpr int kNetFlat = 4 * 4 * 4 * 32;

__host__ __device__ constexpr int net_cin(int l) { return l == 0 ? 2 : 32; }
__host__ __device__ constexpr int net_din(int l) { return kNetG >> l; }   // input edge of conv l

// Offsets (floats) of every tensor in the flat parameter vector.
struct NetLayout {
    long long cw[4], cb[4], f1w, f1b, f2w, f2b, total;
    constexpr NetLayout() : cw{}, cb{}, f1w(0), f1b(0), f2w(0), f2b(0), total(0) {
        long long o = 0;
        for (int l = 0; l < 4; ++l) {
            cw[l] = o;
            o += 32LL * 64 * net_cin(l);
            cb[l] = o;
            o += 32;
        }
        f1w = o;
        o += (long long)kNetHidden * kNetFlat;
        f1b = o;
        o += kNetHidden;
        f2w = o;
        o += (long long)kNetOut * kNetHidden;
        f2b = o;
        o += kNetOut;
        total = o;
    }
};

struct NetPtrs {
    NetLayout L;
    int max_batch;
    float *theta, *grad, *m, *v;   // fp32 parameters, gradients, Adam moments
    uint16_t *wbf[4];              // bf16 conv weights [32][64][Cin]
    uint16_t *wt[4];               // bf16 transposes [Cin][64][32] (layers 1..3)
    uint16_t *x;                   // input [B][64^3][2]
    uint16_t *a[4];                // conv outputs (after ReLU) [B][(32 >> l)^3][32]
    uint16_t *d[4];                // gradients wrt conv pre-activations, same shapes
    float *h, *out, *dh, *dout;    // [B][128], [B][12], [B][128], [B][12]
    float *y;                      // labels [B][6] (pose / limits)
    float *loss;                   // per-step loss log
    int *step;                     // optimiser step counter
    void *samples;                 // synthetic-pair parameters [B]
};

// The plane-staged forward convolution (conv.cu) for 32 input channels:
// whether it applies to an input of edge D, the launch, and its error flag.
bool conv_planes_applies(int D, int Cin);
cudaError_t conv_planes_forward(const uint16_t *X, int batch, int D, const uint16_t *W, const float *bias,
                                uint16_t *Y, cudaStream_t s);
cudaError_t conv_planes_error_flag(unsigned int *out, bool clear);
bool conv_c2_applies(int D, int Cin);
cudaError_t conv_c2_forward(const uint16_t *X, int batch, int D, const uint16_t *W, const float *bias, uint16_t *Y,
                            cudaStream_t s);
cudaError_t conv_planes_wgrad(const uint16_t *X, int batch, int D, const uint16_t *dY, float *dW, cudaStream_t s);
// the plane-staged data gradient of the same convolution (dgrad.cu)
bool dgrad_planes_applies(int D);
cudaError_t dgrad_planes(const uint16_t *dY, int batch, int D, const uint16_t *Wt, const uint16_t *act,
                         uint16_t *dX, cudaStream_t s);
cudaError_t dgrad_planes_error_flag(unsigned int *out, bool clear);

}  // namespace pfreg
