// kernels.h -- launch interfaces between the C-ABI host code and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace pfreg {

constexpr int kMomStride = 12;   // n S1 S2lo S2hi ST T1 T2 0 | n_nn A B C
constexpr int kMaxParticles = 65536;

// Measurement of P matrices (Fig. 1 "measurement"): moments accumulated
// (atomically, integer) into mom[P][12], which the caller zeroes first.
struct MeasureArgs {
    const uint32_t *src_quad;   // image modes: quad-packed source (launch_pack_quads)
    const uint8_t *tgt_img;
    const uint32_t *src_bits;   // mask modes: source mask, 1 bit per voxel
    const uint8_t *tgt_mask;    // mask modes: target mask bytes (0/1)
    const float *mats;          // [P][12]
    unsigned long long *mom;    // [P][12]
    Geometry g;
    int P;
    int rows_per_item;          // target rows per work item
    int n_rowblocks;            // ceil(rows / rows_per_item)
    int items_per_warp;         // tile shape: consecutive work items per warp (0 = default)
    float fdims[4];             // source SX, SX * SY, SY - 2, SZ - 2 as floats (host-filled)
};

// Filter parameters shared by the per-iteration kernels.
struct FilterParams {
    Geometry g;
    int mode;
    int N;
    float lim[6];
    float sigma0_frac, sigma_decay;
    int gamma_log2;
    uint64_t seed;
    uint64_t n_min;             // overlap threshold (voxels)
    uint64_t b_full;            // |T| of the target mask (Dice denominator)
    int log_capacity;
    int estimator;              // pf_estimator
    double sig0[6];             // perturbation base: sigma_kd = sig0_d * decay^k (default
                                // sigma0_frac * L_d; a proposal's spread after pf_seed_gaussian)
};

struct IterLog {
    double est[6];
    double best;
    double ess;
    unsigned long long evals;   // particle-voxel evaluations visited (sum of overlap counts)
    double est_dice;            // Dice of the masks at the estimate (-1 when not traced)
    int32_t best_idx;
    int32_t k;
};

struct FilterBuffers {
    float *poses;               // [6][N] current cloud (resampled)
    float *poses_meas;          // [6][N] cloud measured in the last iteration
    float *mats;                // [N][12]
    unsigned long long *mom;    // [N][12]
    double *scores;             // [N]
    unsigned long long *W;      // [N]
    unsigned long long *C;      // [N] inclusive scan of W
    int32_t *idx;               // [N]
    int32_t *k;                 // iteration counter (device)
    IterLog *log;               // [log_capacity]
    unsigned long long *stats;  // [2] max score (fp64 bits) and evaluation count of the iteration
    float *trace_mat;           // [12] matrix of the estimate (tracing)
    unsigned long long *trace_mom;   // [12] its mask counts (tracing)
    double *quat;               // [4][N] unit quaternion of each measured pose (quaternion estimator)
};

cudaError_t launch_measure(const MeasureArgs &a, bool img, bool mask, cudaStream_t s);
long long measure_items(const MeasureArgs &a);   // work items of one measurement launch
cudaError_t launch_pack_quads(const uint8_t *src, const int32_t dims[3], uint32_t *quad, cudaStream_t s);
int rows_per_item_for(int target_x);
cudaError_t launch_init_particles(const FilterParams &p, const FilterBuffers &b, cudaStream_t s);
cudaError_t launch_seed_gaussian(const FilterParams &p, const FilterBuffers &b, const float mean[6],
                                 const float std[6], cudaStream_t s);
cudaError_t launch_predict(const FilterParams &p, const FilterBuffers &b, cudaStream_t s);
cudaError_t launch_finalise(const FilterParams &p, const FilterBuffers &b, cudaStream_t s);
// Tracing of the estimate (Sec. 3.2: the masks are warped with the estimate
// and their overlap score is taken after every iteration): matrix of the
// last iteration's estimate, then (after a mask measurement) its Dice.
cudaError_t launch_trace_prepare(const FilterParams &p, const FilterBuffers &b, cudaStream_t s);
cudaError_t launch_trace_finish(const FilterParams &p, const FilterBuffers &b, cudaStream_t s);
cudaError_t launch_pack_bits(const uint8_t *mask, int64_t nvox, uint32_t *bits, cudaStream_t s);
cudaError_t launch_count_nonzero(const uint8_t *v, int64_t n, unsigned long long *out, cudaStream_t s);
cudaError_t launch_binarise(const uint8_t *in, uint8_t *out, int64_t n, cudaStream_t s);
cudaError_t launch_pose_matrix(const float *pose, Geometry g, float *mat_out, cudaStream_t s);
cudaError_t launch_score_one(int mode, const unsigned long long *mom, unsigned long long b_full,
                             unsigned long long n_min, double *out, cudaStream_t s);
cudaError_t launch_philox(const uint32_t *ctr_key, uint32_t *out, cudaStream_t s);

struct WarpFrames {
    static constexpr int kMax = 64;
    const uint8_t *in[kMax];
    uint8_t *out[kMax];
};
cudaError_t launch_warp(const WarpFrames &f, int n, const float pose[6], Geometry g, int interp,
                        cudaStream_t s);

// Bounds checks of the debug build (-DPF_DEBUG=1) of the measurement and warp
// kernels: out-of-bounds gather indices seen (the load was skipped), the first
// bad index, whether the checks are compiled in; clear resets the counters.
cudaError_t measure_debug_bounds(bool clear, unsigned long long *hits, long long *first, bool *on);
cudaError_t warp_debug_bounds(bool clear, unsigned long long *hits, long long *first, bool *on);

// One registration of a batch (device table entry): its measurement
// arguments, filter parameters and buffers, and its iteration count.
struct BatchReg {
    MeasureArgs ma;
    FilterParams P;
    FilterBuffers B;
    int32_t n_iters;
    int32_t img, mask;
};

// Batched kernels over many registrations: measurement over the listed
// registrations' concatenated items (offs = item prefix), prediction over all
// particles (poffs = particle prefix), and the update: scores and weights over
// all particles with each registration padded to whole warps (poffs32), then
// one CTA per registration.
// Registrations whose iteration counter has reached n_iters are skipped.
cudaError_t launch_measure_batch(const BatchReg *regs, const int32_t *list, const long long *offs, int nlist,
                                 long long total_items, bool img, bool mask, int items_per_warp, int max_tx,
                                 cudaStream_t s);
constexpr int kDefaultItemsPerWarp = 8;
// Candidate tile shapes (work items per warp) of the autotuner.
constexpr int kTileCandidates[] = {1, 2, 4, 8, 16, 32};
cudaError_t launch_predict_batch(const BatchReg *regs, const long long *poffs, int nregs, long long total,
                                 cudaStream_t s);
cudaError_t launch_finalise_batch(const BatchReg *regs, const long long *poffs32, int nregs, long long total32,
                                  cudaStream_t s);

// Process-wide count of kernel launches issued by this library (launches
// recorded while a CUDA graph is being captured are not counted; each graph
// replay counts its kernels instead).
bool capturing();
void count_launches(uint64_t n);
uint64_t launches();

// Device allocations: every cudaMalloc / cudaMallocAsync of the library goes
// through these, which count the successful ones process-wide.
cudaError_t dev_malloc_bytes(void **p, size_t bytes);
cudaError_t dev_malloc_async_bytes(void **p, size_t bytes, cudaStream_t s);
template <class T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc_bytes(reinterpret_cast<void **>(p), bytes);
}
template <class T>
cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t s) {
    return dev_malloc_async_bytes(reinterpret_cast<void **>(p), bytes, s);
}
uint64_t device_allocs();

}  // namespace pfreg
