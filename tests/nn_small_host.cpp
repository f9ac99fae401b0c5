// The proposal network's CUDA-core kernels -- the weight transpose, the
// fully connected layers and their gradients, the bias gradient, the
// Gaussian loss, Adam, the bf16 weight copies, the uniform initialisation and
// the input's box average -- copied verbatim by the test out of nn.cu into
// nn_small.inc and run block by block on the host under the emulation of
// tests/host_shim/warp_emulation.h.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "host_shim/nn_device.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

namespace pfreg {
namespace nn {
#include "nn_small.inc"
}
}  // namespace pfreg

namespace {
template <class K>
void launch(unsigned blocks, unsigned threads, K &&kernel) {
    gridDim.x = blocks;
    blockDim.x = threads;
    for (unsigned b = 0; b < blocks; ++b) {
        blockIdx.x = b;
        host_warp::run((int)threads, [&](int) { kernel(); });
    }
}
unsigned cover(long long n, unsigned t) { return (unsigned)((n + t - 1) / t); }
}  // namespace

using namespace pfreg::nn;

extern "C" {

void dm_transpose_w(const uint16_t *W, int Cin, uint16_t *Wt) {
    launch(3, 64, [&] { k_transpose_w(W, Cin, Wt); });
}
// in_bf16: the input is bf16 bits (in16), else fp32 (in32)
void dm_fc_forward(int in_bf16, const float *in32, const uint16_t *in16, int B, int K, const float *W,
                   const float *bias, int N, float *out, int relu) {
    launch(cover((long long)B * N * 32, 128), 128, [&] {
        if (in_bf16) k_fc_forward<uint16_t>(in16, B, K, W, bias, N, out, relu);
        else k_fc_forward<float>(in32, B, K, W, bias, N, out, relu);
    });
}
// bf16: the activation and the gradient are bf16 bits (act16, din16), else fp32
void dm_fc_backward_input(int bf16, const float *dout, int B, int N, const float *W, int K, const float *act32,
                          const uint16_t *act16, float *din32, uint16_t *din16) {
    launch(cover((long long)B * K, 96), 96, [&] {
        if (bf16) k_fc_backward_input<uint16_t, uint16_t>(dout, B, N, W, K, act16, din16);
        else k_fc_backward_input<float, float>(dout, B, N, W, K, act32, din32);
    });
}
void dm_fc_backward_weight(int in_bf16, const float *dout, int B, int N, const float *in32, const uint16_t *in16,
                           int K, float *dW, float *db) {
    launch(cover((long long)N * K, 96), 96, [&] {
        if (in_bf16) k_fc_backward_weight<uint16_t>(dout, B, N, in16, K, dW, db);
        else k_fc_backward_weight<float>(dout, B, N, in32, K, dW, db);
    });
}
void dm_bias_grad(const uint16_t *dY, long long rows, int blocks, float *db) {
    launch((unsigned)blocks, 256, [&] { k_bias_grad(dY, rows, db); });
}
void dm_nll(const float *out, const float *y, int B, float *dout, float *loss_log, int step) {
    launch(cover((long long)B * 6, 64), 64, [&] { k_nll(out, y, B, dout, loss_log, &step); });
}
void dm_adam(float *theta, float *m, float *v, const float *g, long long n, float lr, int step) {
    launch(3, 64, [&] { k_adam(theta, m, v, g, n, lr, &step); });
    int s = step;
    launch(1, 32, [&] {
        if (threadIdx.x == 0) k_step_inc(&s);
    });
    if (s != step + 1) std::abort();
}
void dm_to_bf16(const float *a, long long n, uint16_t *out) {
    launch(3, 64, [&] { k_to_bf16(a, n, out); });
}
void dm_init_uniform(float *p, long long n, float a, uint64_t seed, uint32_t tensor) {
    launch(3, 64, [&] { k_init_uniform(p, n, a, seed, tensor); });
}
void dm_downsample(const uint8_t *vol, const int32_t dims[3], const float origin[3], const float spacing[3],
                   const float box_o[3], const float h[3], int G, int c, uint16_t *x) {
    DownArgs a{};
    a.vol = vol;
    for (int d = 0; d < 3; ++d) {
        a.dims[d] = dims[d];
        a.origin[d] = origin[d];
        a.spacing[d] = spacing[d];
        a.box_o[d] = box_o[d];
        a.h[d] = h[d];
    }
    a.G = G;
    a.c = c;
    a.x = x;
    launch(cover((long long)G * G * G, 256), 256, [&] { k_downsample(a); });
}
}
