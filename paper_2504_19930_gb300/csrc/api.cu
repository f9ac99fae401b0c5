// api.cu -- the C ABI declared in include/pfreg.h.
//
// Host code here only validates arguments, owns device memory, moves bytes
// and launches kernels; every arithmetic step of the registration runs in the
// kernels of measure.cu, filter.cu and warp.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <map>
#include <atomic>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pfreg.h"
#include "kernels.h"

using namespace pfreg;

namespace {
// NVTX range around a host call (shows the library's steps on a profiler's
// timeline; costs nothing when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

namespace {

thread_local std::string g_err;
thread_local bool g_capturing = false;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                   \
    } while (0)

constexpr float kHalfPi = 1.57079637f;   // fp32 rounding of pi/2 (>= pi/2)
constexpr int kMaxDim = 2048;
constexpr size_t kMaxSourceVoxels = (size_t)1 << 28;   // 32-bit gather indices into the packed copy
constexpr size_t kMaxTargetVoxels = (size_t)1 << 26;   // keeps n * S2 within 128 bits
constexpr int kLogCapacity = 4096;

bool finite3(const float v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int check_volume(const pf_volume *v, const char *name) {
    if (!v) return fail(PF_EINVAL, "%s is NULL", name);
    if (!v->data) return fail(PF_EINVAL, "%s->data is NULL", name);
    for (int d = 0; d < 3; ++d)
        if (v->dims[d] < 2 || v->dims[d] > kMaxDim)
            return fail(PF_EINVAL, "%s dims[%d] = %d outside [2, %d]", name, d, v->dims[d], kMaxDim);
    if (!finite3(v->origin)) return fail(PF_EINVAL, "%s origin is not finite", name);
    for (int d = 0; d < 3; ++d)
        if (!(v->spacing[d] > 0.0f && v->spacing[d] <= 1e6f))
            return fail(PF_EINVAL, "%s spacing[%d] = %g outside (0, 1e6]", name, d, (double)v->spacing[d]);
    return PF_OK;
}

// Spacing argument of the plain-array entry points: NULL means 1.
bool spacing_ok(const float *s) {
    if (!s) return true;
    for (int d = 0; d < 3; ++d)
        if (!(s[d] > 0.0f && s[d] <= 1e6f)) return false;
    return true;
}

size_t nvox(const int32_t d[3]) { return (size_t)d[0] * d[1] * d[2]; }

bool same_grid(const pf_volume *a, const pf_volume *b) {
    for (int d = 0; d < 3; ++d)
        if (a->dims[d] != b->dims[d] || a->origin[d] != b->origin[d] || a->spacing[d] != b->spacing[d])
            return false;
    return true;
}

int check_config(const pf_config *c) {
    if (!c) return fail(PF_EINVAL, "cfg is NULL");
    if (c->mode < PF_MASK_DICE || c->mode > PF_COMBINED) return fail(PF_EINVAL, "mode %d unknown", c->mode);
    if (c->n_particles < 1 || c->n_particles > kMaxParticles)
        return fail(PF_EINVAL, "n_particles %d outside [1, %d]", c->n_particles, kMaxParticles);
    for (int d = 0; d < 3; ++d) {
        if (!(c->rot_limit[d] > 0.0f && c->rot_limit[d] <= kHalfPi))
            return fail(PF_EINVAL, "rot_limit[%d] = %g outside (0, pi/2]", d, (double)c->rot_limit[d]);
        if (!(c->trans_limit[d] > 0.0f && c->trans_limit[d] <= 2048.0f))
            return fail(PF_EINVAL, "trans_limit[%d] = %g outside (0, 2048]", d, (double)c->trans_limit[d]);
    }
    if (!(c->sigma0_frac > 0.0f && c->sigma0_frac <= 1.0f)) return fail(PF_EINVAL, "sigma0_frac outside (0, 1]");
    if (!(c->sigma_decay > 0.0f && c->sigma_decay <= 1.0f)) return fail(PF_EINVAL, "sigma_decay outside (0, 1]");
    if (c->gamma_log2 < 0 || c->gamma_log2 > 10) return fail(PF_EINVAL, "gamma_log2 outside [0, 10]");
    if (!(c->min_overlap_frac >= 0.0f && c->min_overlap_frac <= 1.0f))
        return fail(PF_EINVAL, "min_overlap_frac outside [0, 1]");
    if (c->estimator != PF_EST_MEAN && c->estimator != PF_EST_QUATERNION)
        return fail(PF_EINVAL, "estimator %d unknown", c->estimator);
    if (c->autotune != 0 && c->autotune != 1) return fail(PF_EINVAL, "autotune must be 0 or 1");
    return PF_OK;
}

// Device copy of a volume description's bytes (into dst, n bytes).
cudaError_t copy_in(void *dst, const pf_volume *v, size_t n, cudaStream_t s) {
    return cudaMemcpyAsync(dst, v->data, n, v->is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
}

Geometry make_geometry(const int32_t sd[3], const float so[3], const float *ss, const int32_t td[3],
                       const float to[3], const float *ts) {
    Geometry g;
    for (int d = 0; d < 3; ++d) {
        g.sd[d] = sd[d];
        g.td[d] = td[d];
        g.so[d] = so[d];
        g.to[d] = to[d];
        g.ss[d] = ss ? ss[d] : 1.0f;
        g.ts[d] = ts ? ts[d] : 1.0f;
        // a = (c - o_T) / s_T with c = o_S + s_S (dims_S - 1)/2: fp64, one rounding
        const double c = (double)so[d] + (double)g.ss[d] * ((double)(sd[d] - 1) / 2.0);
        g.a[d] = (float)((c - (double)to[d]) / (double)g.ts[d]);
    }
    return g;
}

}  // namespace

namespace pfreg {
bool capturing() { return g_capturing; }
}  // namespace pfreg

// Host-side fault injection: a cap on the device bytes one context may
// allocate (pf_debug_alloc_limit); beyond it the allocation reports
// cudaErrorMemoryAllocation without calling cudaMalloc.  0 = no cap.
static std::atomic<long long> g_alloc_limit{0};

struct pf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    pf_config cfg{};
    FilterParams P{};
    FilterBuffers B{};
    MeasureArgs MA{};
    bool img = false, mask = false, trace = false;
    uint8_t *tgt_img = nullptr, *tgt_mask = nullptr;
    uint32_t *src_quad = nullptr;
    uint32_t *src_bits = nullptr;
    unsigned long long *d_u64 = nullptr;   // small scratch: counts
    double *d_score = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // timing of the measurement kernel inside the iteration graph: two event
    // record nodes around it whose events are swapped per launch
    cudaEvent_t ev_before = nullptr, ev_after = nullptr;
    cudaGraphNode_t node_before = nullptr, node_after = nullptr;
    uint64_t graph_kernels = 0;             // kernel nodes of one iteration's graph
    std::vector<cudaEvent_t> prof_events;   // 2 per timed iteration
    int prof_next = 0;
    bool prof_default = true;               // the record nodes hold ev_before/ev_after
    // scratch for pf_measure_matrices / the estimate's score
    float *x_mats = nullptr;
    unsigned long long *x_mom = nullptr;
    int x_cap = 0;
    std::vector<void *> allocs;

    long long alloc_bytes = 0;
    // One device block that alloc() carves the context's buffers from (one
    // cudaMalloc instead of one per buffer: creation lies inside the time of
    // every registration, and a 64^3 one takes under 2 ms).
    char *arena = nullptr;
    size_t arena_cap = 0, arena_used = 0;

    static size_t padded(size_t bytes) { return ((bytes > 0 ? bytes : 1) + 255) & ~(size_t)255; }

    cudaError_t raw_alloc(void **q, size_t bytes) {
        const long long cap = g_alloc_limit.load();
        if (cap > 0 && alloc_bytes + (long long)bytes > cap) return cudaErrorMemoryAllocation;
        cudaError_t e = dev_malloc(q, bytes);
        if (e == cudaSuccess) {
            allocs.push_back(*q);
            alloc_bytes += (long long)bytes;
        }
        return e;
    }
    cudaError_t reserve(size_t bytes) {
        void *q = nullptr;
        cudaError_t e = raw_alloc(&q, bytes);
        if (e == cudaSuccess) {
            arena = static_cast<char *>(q);
            arena_cap = bytes;
            arena_used = 0;
        }
        return e;
    }
    // count elements of T, 256-byte aligned; from the block while it has room
    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        const size_t bytes = padded(count * sizeof(T));
        if (arena && arena_cap - arena_used >= bytes) {
            *p = reinterpret_cast<T *>(arena + arena_used);
            arena_used += bytes;
            return cudaSuccess;
        }
        void *q = nullptr;
        cudaError_t e = raw_alloc(&q, bytes);
        if (e == cudaSuccess) *p = static_cast<T *>(q);
        return e;
    }
    ~pf_ctx() {
        if (exec) cudaGraphExecDestroy(exec);
        for (cudaEvent_t e : prof_events) cudaEventDestroy(e);
        if (ev_before) cudaEventDestroy(ev_before);
        if (ev_after) cudaEventDestroy(ev_after);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (void *p : allocs) cudaFree(p);
        if (x_mats) cudaFree(x_mats);
        if (x_mom) cudaFree(x_mom);
    }
};

namespace {

int ensure_scratch(pf_ctx *c, int M) {
    if (M <= c->x_cap) return PF_OK;
    if (c->x_mats) cudaFree(c->x_mats);
    if (c->x_mom) cudaFree(c->x_mom);
    c->x_mats = nullptr;
    c->x_mom = nullptr;
    c->x_cap = 0;
    CU(dev_malloc(&c->x_mats, sizeof(float) * 12 * (size_t)M));
    CU(dev_malloc(&c->x_mom, sizeof(unsigned long long) * kMomStride * (size_t)M));
    c->x_cap = M;
    return PF_OK;
}

// Measurement of M matrices already in c->x_mats into c->x_mom (zeroed here).
int measure_scratch(pf_ctx *c, int M, const float a[3]) {
    CU(cudaMemsetAsync(c->x_mom, 0, sizeof(unsigned long long) * kMomStride * (size_t)M, c->stream));
    MeasureArgs ma = c->MA;
    ma.mats = c->x_mats;
    ma.mom = c->x_mom;
    ma.P = M;
    for (int d = 0; d < 3; ++d) ma.g.a[d] = a[d];
    CU(launch_measure(ma, c->img, c->mask, c->stream));
    return PF_OK;
}

// One filter iteration as a CUDA graph: predict -> measure -> finalise, with
// event-record nodes around the measurement kernel (for pf_profile_*).
int build_graph(pf_ctx *c) {
    CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CU(cudaEventCreate(&c->ev_before));
    CU(cudaEventCreate(&c->ev_after));
    g_capturing = true;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t es[6];
        es[0] = launch_predict(c->P, c->B, c->cap_stream);
        es[1] = cudaEventRecordWithFlags(c->ev_before, c->cap_stream, cudaEventRecordExternal);
        es[2] = launch_measure(c->MA, c->img, c->mask, c->cap_stream);
        es[3] = cudaEventRecordWithFlags(c->ev_after, c->cap_stream, cudaEventRecordExternal);
        es[4] = launch_finalise(c->P, c->B, c->cap_stream);
        if (c->trace) {   // the estimate's mask Dice, logged every iteration
            MeasureArgs tm = c->MA;
            tm.mats = c->B.trace_mat;
            tm.mom = c->B.trace_mom;
            tm.P = 1;
            cudaError_t t1 = launch_trace_prepare(c->P, c->B, c->cap_stream);
            cudaError_t t2 = launch_measure(tm, false, true, c->cap_stream);
            cudaError_t t3 = launch_trace_finish(c->P, c->B, c->cap_stream);
            es[4] = es[4] != cudaSuccess ? es[4] : t1 != cudaSuccess ? t1 : t2 != cudaSuccess ? t2 : t3;
        }
        es[5] = cudaStreamEndCapture(c->cap_stream, &c->graph);
        for (cudaError_t x : es)
            if (x != cudaSuccess && e == cudaSuccess) e = x;
    }
    g_capturing = false;
    if (e != cudaSuccess) return fail(PF_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    size_t n = 0;
    CU(cudaGraphGetNodes(c->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CU(cudaGraphGetNodes(c->graph, nodes.data(), &n));
    c->graph_kernels = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        CU(cudaGraphNodeGetType(nd, &t));
        c->graph_kernels += t == cudaGraphNodeTypeKernel;
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        CU(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        if (ev == c->ev_before) c->node_before = nd;
        if (ev == c->ev_after) c->node_after = nd;
    }
    if (!c->node_before || !c->node_after) return fail(PF_ECUDA, "timing nodes not found in the graph");
    CU(cudaGraphInstantiate(&c->exec, c->graph, 0));
    return PF_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the measurement's tile shape (work items per warp).  Every
// candidate gives the same moments bit for bit (integer atomics), so the
// choice only moves time: each candidate measures the context's current
// cloud (one warm-up and two timed launches, CUDA events) and the fastest
// wins.  Results are cached per (mode, source dims, target dims, N) for the
// process, so contexts of a repeated shape pay the search once.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;

std::string tune_key(const pf_ctx *c) {
    char buf[160];
    snprintf(buf, sizeof buf, "%d%d|%d,%d,%d|%d,%d,%d|%d", (int)c->img, (int)c->mask, c->MA.g.sd[0], c->MA.g.sd[1],
             c->MA.g.sd[2], c->MA.g.td[0], c->MA.g.td[1], c->MA.g.td[2], c->P.N);
    return buf;
}

// Time `launch(ipw)` for every candidate; returns the fastest (ms in *best_ms).
template <class F>
int time_candidates(cudaStream_t s, F launch, int *best, float *best_ms) {
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    *best = kDefaultItemsPerWarp;
    *best_ms = 1e30f;
    int rc = PF_OK;
    for (int cand : kTileCandidates) {
        cudaError_t e = launch(cand);   // warm-up
        float tmin = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch(cand);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < tmin) tmin = ms;
        }
        if (e != cudaSuccess) {
            rc = fail(PF_ECUDA, "autotune: %s", cudaGetErrorString(e));
            break;
        }
        if (tmin < *best_ms) {
            *best_ms = tmin;
            *best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// Pick the context's tile shape (iteration 0: the prediction only builds the
// matrices of the initial cloud and zeroes the moments, so it can run here).
int autotune_ctx(pf_ctx *c) {
    const std::string key = tune_key(c);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            c->MA.items_per_warp = it->second;
            return PF_OK;
        }
    }
    CU(launch_predict(c->P, c->B, c->stream));
    int best = kDefaultItemsPerWarp;
    float ms = 0.0f;
    int rc = time_candidates(c->stream, [&](int ipw) {
        MeasureArgs ma = c->MA;
        ma.items_per_warp = ipw;
        return launch_measure(ma, c->img, c->mask, c->stream);
    }, &best, &ms);
    if (rc) return rc;
    CU(cudaMemsetAsync(c->B.mom, 0, sizeof(unsigned long long) * kMomStride * (size_t)c->P.N, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->MA.items_per_warp = best;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    return PF_OK;
}

// Re-capture the iteration graph after the filter parameters changed.
int rebuild_graph(pf_ctx *c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->ev_before) cudaEventDestroy(c->ev_before);
    if (c->ev_after) cudaEventDestroy(c->ev_after);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->exec = nullptr;
    c->graph = nullptr;
    c->ev_before = c->ev_after = nullptr;
    c->cap_stream = nullptr;
    c->node_before = c->node_after = nullptr;
    c->prof_default = true;
    return build_graph(c);
}

int set_record_events(pf_ctx *c, cudaEvent_t before, cudaEvent_t after) {
    CU(cudaGraphExecEventRecordNodeSetEvent(c->exec, c->node_before, before));
    CU(cudaGraphExecEventRecordNodeSetEvent(c->exec, c->node_after, after));
    return PF_OK;
}

}  // namespace

extern "C" {

void pf_config_default(pf_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->mode = PF_MASK_DICE;
    cfg->n_particles = 256;
    for (int d = 0; d < 3; ++d) {
        cfg->rot_limit[d] = 0.2617994f;   // 15 degrees
        cfg->trans_limit[d] = 8.0f;
    }
    cfg->sigma0_frac = 0.25f;
    cfg->sigma_decay = 0.8f;
    cfg->gamma_log2 = 5;
    cfg->seed = 0;
    cfg->min_overlap_frac = 0.01f;
    cfg->trace_estimate = 0;
    cfg->estimator = PF_EST_MEAN;
}

const char *pf_last_error(void) { return g_err.c_str(); }

uint64_t pf_kernel_launches(void) { return launches(); }

uint64_t pf_debug_device_allocs(void) { return device_allocs(); }

int pf_debug_bounds(int32_t clear, int32_t *checks_on, uint64_t *hits, int64_t *first_bad) {
    if (!checks_on || !hits || !first_bad) return fail(PF_EINVAL, "NULL argument");
    CU(cudaDeviceSynchronize());
    unsigned long long h1 = 0, h2 = 0;
    long long f1 = 0, f2 = 0;
    bool on1 = false, on2 = false;
    CU(measure_debug_bounds(clear != 0, &h1, &f1, &on1));
    CU(warp_debug_bounds(clear != 0, &h2, &f2, &on2));
    *checks_on = (on1 && on2) ? 1 : 0;
    *hits = h1 + h2;
    *first_bad = h1 ? f1 : f2;
    return PF_OK;
}

int pf_register_init(pf_ctx **out, const pf_volume *src, const pf_volume *tgt, const pf_volume *src_mask,
                     const pf_volume *tgt_mask, const pf_config *cfg, void *cuda_stream) {
    NvtxRange nvtx("pf_register_init");
    if (!out) return fail(PF_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc) return rc;
    const bool img = cfg->mode == PF_IMAGE_NCC || cfg->mode == PF_COMBINED;
    const bool mask = cfg->mode != PF_IMAGE_NCC;
    if (img) {
        if ((rc = check_volume(src, "src")) || (rc = check_volume(tgt, "tgt"))) return rc;
    }
    if (mask) {
        if ((rc = check_volume(src_mask, "src_mask")) || (rc = check_volume(tgt_mask, "tgt_mask"))) return rc;
    }
    if (img && mask && (!same_grid(src, src_mask) || !same_grid(tgt, tgt_mask)))
        return fail(PF_EINVAL, "combined mode: each mask must share its image's dims and origin");
    // Image mode may carry the masks too, for tracing the estimate's Dice.
    const bool have_masks = mask || (src_mask != nullptr && tgt_mask != nullptr);
    if (img && !mask && have_masks) {
        if ((rc = check_volume(src_mask, "src_mask")) || (rc = check_volume(tgt_mask, "tgt_mask"))) return rc;
        if (!same_grid(src, src_mask) || !same_grid(tgt, tgt_mask))
            return fail(PF_EINVAL, "tracing masks must share their image's dims and origin");
    }
    if (cfg->trace_estimate && !have_masks)
        return fail(PF_EINVAL, "trace_estimate needs src_mask and tgt_mask");
    const pf_volume *S = img ? src : src_mask;
    const pf_volume *T = img ? tgt : tgt_mask;
    if (nvox(S->dims) > kMaxSourceVoxels) return fail(PF_EINVAL, "source has more than 2^28 voxels");
    if (nvox(T->dims) > kMaxTargetVoxels) return fail(PF_EINVAL, "target has more than 2^26 voxels");

    pf_ctx *c = new (std::nothrow) pf_ctx();
    if (!c) return fail(PF_ENOMEM, "host allocation failed");
    auto bail = [&](int code) {
        delete c;
        return code;
    };
#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "%s: %s", #call, \
                             cudaGetErrorString(e_)));                                        \
    } while (0)

    CK(cudaGetDevice(&c->device));
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->cfg = *cfg;
    c->img = img;
    c->mask = mask;
    c->trace = cfg->trace_estimate != 0;
    const int N = cfg->n_particles;
    const Geometry g = make_geometry(S->dims, S->origin, S->spacing, T->dims, T->origin, T->spacing);
    const size_t ns = nvox(S->dims), nt = nvox(T->dims);

    FilterParams &P = c->P;
    P.g = g;
    P.mode = cfg->mode;
    P.N = N;
    for (int d = 0; d < 3; ++d) {
        P.lim[d] = cfg->rot_limit[d];
        P.lim[3 + d] = cfg->trans_limit[d];
    }
    P.sigma0_frac = cfg->sigma0_frac;
    for (int d = 0; d < 6; ++d) P.sig0[d] = (double)cfg->sigma0_frac * (double)P.lim[d];   // exact product
    P.sigma_decay = cfg->sigma_decay;
    P.gamma_log2 = cfg->gamma_log2;
    P.seed = cfg->seed;
    P.n_min = (uint64_t)((double)cfg->min_overlap_frac * (double)nt);
    P.b_full = 0;
    P.log_capacity = kLogCapacity;
    P.estimator = cfg->estimator;

    FilterBuffers &B = c->B;
    uint8_t *tmp = nullptr;   // staging of host masks
    const bool host_masks = have_masks && (!src_mask->is_device || !tgt_mask->is_device);
    // Every device buffer of the context, listed once: the list is walked to
    // size the block, then again to carve the buffers from it.
    auto buffers = [&](auto &&take) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        auto want = [&](auto **p, size_t n) {
            if (e == cudaSuccess) e = take(p, n);
        };
        want(&B.poses, 6 * (size_t)N);
        want(&B.poses_meas, 6 * (size_t)N);
        want(&B.mats, 12 * (size_t)N);
        want(&B.mom, (size_t)kMomStride * N);
        want(&B.scores, (size_t)N);
        want(&B.W, (size_t)N);
        want(&B.C, (size_t)N);
        want(&B.idx, (size_t)N);
        want(&B.k, 1);
        want(&B.log, (size_t)kLogCapacity);
        if (P.estimator == PF_EST_QUATERNION) want(&B.quat, 4 * (size_t)N);
        want(&c->d_u64, 4);
        want(&c->d_score, 1);
        if (img) {
            want(&c->src_quad, ns);
            want(&c->tgt_img, nt);
        }
        want(&B.stats, 2);
        want(&B.trace_mat, 12);
        want(&B.trace_mom, (size_t)kMomStride);
        if (have_masks) {
            want(&c->src_bits, (ns + 31) / 32);
            want(&c->tgt_mask, nt);
            if (host_masks) want(&tmp, ns > nt ? ns : nt);
        }
        return e;
    };
    size_t block = 0;
    buffers([&](auto **p, size_t n) {
        block += pf_ctx::padded(n * sizeof(**p));
        return cudaSuccess;
    });
    CK(c->reserve(block));
    CK(buffers([&](auto **p, size_t n) { return c->alloc(p, n); }));

    if (img) {
        uint8_t *raw = nullptr;
        const uint8_t *sp = static_cast<const uint8_t *>(src->data);
        if (!src->is_device) {
            CK(dev_malloc_async(&raw, ns, c->stream));
            CK(copy_in(raw, src, ns, c->stream));
            sp = raw;
        }
        CK(launch_pack_quads(sp, S->dims, c->src_quad, c->stream));
        if (raw) CK(cudaFreeAsync(raw, c->stream));
        CK(copy_in(c->tgt_img, tgt, nt, c->stream));
    }
    if (have_masks) {
        const uint8_t *sm = static_cast<const uint8_t *>(src_mask->data);
        const uint8_t *tm = static_cast<const uint8_t *>(tgt_mask->data);
        if (!src_mask->is_device) {
            CK(copy_in(tmp, src_mask, ns, c->stream));
            sm = tmp;
        }
        CK(launch_pack_bits(sm, (int64_t)ns, c->src_bits, c->stream));
        if (!tgt_mask->is_device) {
            CK(cudaStreamSynchronize(c->stream));   // tmp is reused for the target
            CK(copy_in(tmp, tgt_mask, nt, c->stream));
            tm = tmp;
        }
        CK(launch_binarise(tm, c->tgt_mask, (int64_t)nt, c->stream));
        CK(cudaMemsetAsync(c->d_u64, 0, sizeof(unsigned long long), c->stream));
        CK(launch_count_nonzero(c->tgt_mask, (int64_t)nt, c->d_u64, c->stream));
    }

    MeasureArgs &MA = c->MA;
    MA.src_quad = c->src_quad;
    MA.tgt_img = c->tgt_img;
    MA.src_bits = c->src_bits;
    MA.tgt_mask = c->tgt_mask;
    MA.mats = B.mats;
    MA.mom = B.mom;
    MA.g = g;
    MA.P = N;
    MA.rows_per_item = rows_per_item_for(g.td[0]);
    MA.n_rowblocks = (g.td[1] * g.td[2] + MA.rows_per_item - 1) / MA.rows_per_item;
    MA.items_per_warp = kDefaultItemsPerWarp;
    MA.fdims[0] = (float)g.sd[0];
    MA.fdims[1] = (float)((int64_t)g.sd[0] * g.sd[1]);
    MA.fdims[2] = (float)(g.sd[1] - 2);
    MA.fdims[3] = (float)(g.sd[2] - 2);

    CK(cudaMemsetAsync(B.k, 0, sizeof(int32_t), c->stream));
    CK(cudaMemsetAsync(B.mom, 0, sizeof(unsigned long long) * kMomStride * (size_t)N, c->stream));
    CK(launch_init_particles(P, B, c->stream));   // the initial cloud does not depend on b_full
    unsigned long long bfull = 0;
    if (have_masks) CK(cudaMemcpyAsync(&bfull, c->d_u64, sizeof bfull, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));   // one wait for all the set-up work
    P.b_full = bfull;
    if (cfg->autotune) {
        rc = autotune_ctx(c);
        if (rc) return bail(rc);
    }
    rc = build_graph(c);
    if (rc) return bail(rc);
#undef CK
    *out = c;
    return PF_OK;
}

int pf_seed_gaussian(pf_ctx *c, const float mean[6], const float std[6]) {
    if (!c || !mean || !std) return fail(PF_EINVAL, "NULL argument");
    for (int d = 0; d < 6; ++d) {
        if (!std::isfinite(mean[d])) return fail(PF_EINVAL, "mean[%d] is not finite", d);
        if (!(std[d] > 0.0f && std[d] <= 1e6f)) return fail(PF_EINVAL, "std[%d] outside (0, 1e6]", d);
    }
    int32_t k = 0;
    CU(cudaMemcpyAsync(&k, c->B.k, sizeof k, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (k != 0) return fail(PF_ESTATE, "pf_seed_gaussian after the first iteration (k = %d)", k);
    if (c->prof_events.size()) return fail(PF_ESTATE, "pf_seed_gaussian while profiling is armed");
    for (int d = 0; d < 6; ++d) c->P.sig0[d] = (double)std[d];
    CU(launch_seed_gaussian(c->P, c->B, mean, std, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return rebuild_graph(c);
}

int pf_step(pf_ctx *c, int32_t n_iters) {
    NvtxRange nvtx("pf_step");
    if (!c) return fail(PF_EINVAL, "ctx is NULL");
    if (n_iters < 0) return fail(PF_EINVAL, "n_iters < 0");
    for (int32_t i = 0; i < n_iters; ++i) {
        const int slot = c->prof_next;
        if (2 * slot + 1 < (int)c->prof_events.size()) {
            int rc = set_record_events(c, c->prof_events[2 * slot], c->prof_events[2 * slot + 1]);
            if (rc) return rc;
            c->prof_default = false;
            ++c->prof_next;
        } else if (!c->prof_default) {
            int rc = set_record_events(c, c->ev_before, c->ev_after);
            if (rc) return rc;
            c->prof_default = true;
        }
        CU(cudaGraphLaunch(c->exec, c->stream));
        count_launches(c->graph_kernels);
    }
    return PF_OK;
}

int pf_step_measure(pf_ctx *c, int32_t p_begin, int32_t p_end) {
    NvtxRange nvtx("pf_step_measure");
    if (!c) return fail(PF_EINVAL, "ctx is NULL");
    if (p_begin < 0 || p_end < p_begin || p_end > c->P.N)
        return fail(PF_EINVAL, "slice [%d, %d) outside [0, %d]", p_begin, p_end, c->P.N);
    CU(launch_predict(c->P, c->B, c->stream));
    if (p_end > p_begin) {
        MeasureArgs ma = c->MA;
        ma.mats = c->B.mats + 12 * (size_t)p_begin;
        ma.mom = c->B.mom + kMomStride * (size_t)p_begin;
        ma.P = p_end - p_begin;
        CU(launch_measure(ma, c->img, c->mask, c->stream));
    }
    return PF_OK;
}

int pf_step_update(pf_ctx *c) {
    NvtxRange nvtx("pf_step_update");
    if (!c) return fail(PF_EINVAL, "ctx is NULL");
    CU(launch_finalise(c->P, c->B, c->stream));
    if (c->trace) {
        MeasureArgs tm = c->MA;
        tm.mats = c->B.trace_mat;
        tm.mom = c->B.trace_mom;
        tm.P = 1;
        CU(launch_trace_prepare(c->P, c->B, c->stream));
        CU(launch_measure(tm, false, true, c->stream));
        CU(launch_trace_finish(c->P, c->B, c->stream));
    }
    return PF_OK;
}

int pf_moments_device(pf_ctx *c, uint64_t **moments, int64_t *n_words) {
    if (!c || !moments || !n_words) return fail(PF_EINVAL, "NULL argument");
    *moments = reinterpret_cast<uint64_t *>(c->B.mom);
    *n_words = (int64_t)kMomStride * c->P.N;
    return PF_OK;
}

int pf_profile_begin(pf_ctx *c, int32_t capacity) {
    if (!c) return fail(PF_EINVAL, "ctx is NULL");
    if (capacity < 0 || capacity > (1 << 16)) return fail(PF_EINVAL, "capacity outside [0, 65536]");
    CU(cudaStreamSynchronize(c->stream));
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    c->prof_events.clear();
    c->prof_next = 0;
    for (int32_t i = 0; i < 2 * capacity; ++i) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        c->prof_events.push_back(e);
    }
    return PF_OK;
}

int pf_profile_end(pf_ctx *c, double *total_ms, int32_t *n_timed) {
    if (!c || !total_ms || !n_timed) return fail(PF_EINVAL, "NULL argument");
    CU(cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    for (int i = 0; i < c->prof_next; ++i) {
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, c->prof_events[2 * i], c->prof_events[2 * i + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *n_timed = c->prof_next;
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    c->prof_events.clear();
    c->prof_next = 0;
    return PF_OK;
}

int pf_get_iteration(pf_ctx *c, int32_t *k_out) {
    if (!c || !k_out) return fail(PF_EINVAL, "NULL argument");
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaMemcpy(k_out, c->B.k, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return PF_OK;
}

int pf_estimate(pf_ctx *c, float pose_out[6], double *score_out) {
    NvtxRange nvtx("pf_estimate");
    if (!c || !pose_out) return fail(PF_EINVAL, "NULL argument");
    int32_t k = 0;
    int rc = pf_get_iteration(c, &k);
    if (rc) return rc;
    if (k <= 0) return fail(PF_ESTATE, "no iteration has run yet");
    IterLog L;
    CU(cudaMemcpy(&L, c->B.log + ((k - 1) % kLogCapacity), sizeof L, cudaMemcpyDeviceToHost));
    for (int d = 0; d < 6; ++d) pose_out[d] = (float)L.est[d];
    if (score_out) {
        if ((rc = ensure_scratch(c, 1))) return rc;
        float *d_pose = reinterpret_cast<float *>(c->x_mom);   // 6 floats of staging
        CU(cudaMemcpyAsync(d_pose, pose_out, sizeof(float) * 6, cudaMemcpyHostToDevice, c->stream));
        CU(launch_pose_matrix(d_pose, c->P.g, c->x_mats, c->stream));
        if ((rc = measure_scratch(c, 1, c->P.g.a))) return rc;
        CU(launch_score_one(c->P.mode, c->x_mom, c->P.b_full, c->P.n_min, c->d_score, c->stream));
        CU(cudaMemcpyAsync(score_out, c->d_score, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return PF_OK;
}

int pf_get_state(pf_ctx *c, float *poses_measured, uint64_t *moments, double *scores, uint64_t *weights,
                 int32_t *resample_idx, float *poses_next) {
    if (!c) return fail(PF_EINVAL, "ctx is NULL");
    const size_t N = (size_t)c->P.N;
    CU(cudaStreamSynchronize(c->stream));
    if (poses_measured) CU(cudaMemcpy(poses_measured, c->B.poses_meas, 6 * N * sizeof(float), cudaMemcpyDeviceToHost));
    if (moments) CU(cudaMemcpy(moments, c->B.mom, kMomStride * N * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (scores) CU(cudaMemcpy(scores, c->B.scores, N * sizeof(double), cudaMemcpyDeviceToHost));
    if (weights) CU(cudaMemcpy(weights, c->B.W, N * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (resample_idx) CU(cudaMemcpy(resample_idx, c->B.idx, N * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (poses_next) CU(cudaMemcpy(poses_next, c->B.poses, 6 * N * sizeof(float), cudaMemcpyDeviceToHost));
    return PF_OK;
}

int pf_set_state(pf_ctx *c, const float *poses6xN, int32_t k) {
    if (!c || !poses6xN) return fail(PF_EINVAL, "NULL argument");
    if (k < 0) return fail(PF_EINVAL, "k < 0");
    const int N = c->P.N;
    for (int d = 0; d < 6; ++d)
        for (int i = 0; i < N; ++i) {
            const float v = poses6xN[(size_t)d * N + i];
            if (!std::isfinite(v) || v > c->P.lim[d] || v < -c->P.lim[d])
                return fail(PF_EINVAL, "pose[%d][%d] = %g outside the limits", d, i, (double)v);
        }
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaMemcpy(c->B.poses, poses6xN, 6 * (size_t)N * sizeof(float), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->B.k, &k, sizeof k, cudaMemcpyHostToDevice));
    return PF_OK;
}

int pf_get_log(pf_ctx *c, double *est, double *best, double *ess, uint64_t *evals, double *est_dice,
               int32_t *count_inout) {
    if (!c || !count_inout) return fail(PF_EINVAL, "NULL argument");
    int32_t k = 0;
    int rc = pf_get_iteration(c, &k);
    if (rc) return rc;
    int32_t n = *count_inout;
    if (n < 0) n = 0;
    if (n > k) n = k;
    if (n > kLogCapacity) n = kLogCapacity;
    std::vector<IterLog> L(kLogCapacity);
    CU(cudaMemcpy(L.data(), c->B.log, sizeof(IterLog) * kLogCapacity, cudaMemcpyDeviceToHost));
    for (int32_t r = 0; r < n; ++r) {
        const IterLog &e = L[(k - n + r) % kLogCapacity];
        if (est)
            for (int d = 0; d < 6; ++d) est[6 * r + d] = e.est[d];
        if (best) best[r] = e.best;
        if (ess) ess[r] = e.ess;
        if (evals) evals[r] = e.evals;
        if (est_dice) est_dice[r] = e.est_dice;
    }
    *count_inout = n;
    return PF_OK;
}

int pf_measure_matrices(pf_ctx *c, const float *mats, int32_t M, const float a[3], uint64_t *moments_out) {
    if (!c || !mats || !a || !moments_out) return fail(PF_EINVAL, "NULL argument");
    if (M < 1 || M > (1 << 20)) return fail(PF_EINVAL, "M = %d outside [1, 2^20]", M);
    for (size_t i = 0; i < 12 * (size_t)M; ++i)
        if (!std::isfinite(mats[i])) return fail(PF_EINVAL, "matrix entry %zu is not finite", i);
    if (!finite3(a)) return fail(PF_EINVAL, "a is not finite");
    int rc = ensure_scratch(c, M);
    if (rc) return rc;
    // The measurement kernel relies on no offset b being -0 (then no sample
    // coordinate is -0); b + 0 turns -0 into +0 and leaves every other value.
    std::vector<float> m(mats, mats + 12 * (size_t)M);
    for (size_t i = 0; i < (size_t)M; ++i)
        for (int r = 0; r < 3; ++r) m[12 * i + 4 * r + 3] += 0.0f;
    CU(cudaMemcpyAsync(c->x_mats, m.data(), sizeof(float) * 12 * (size_t)M, cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));   // m is released on return
    if ((rc = measure_scratch(c, M, a))) return rc;
    CU(cudaMemcpyAsync(moments_out, c->x_mom, sizeof(uint64_t) * kMomStride * (size_t)M,
                       cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return PF_OK;
}

int pf_register_destroy(pf_ctx *c) {
    if (!c) return PF_OK;
    cudaStreamSynchronize(c->stream);
    delete c;
    return PF_OK;
}

int pf_pose_matrix(const float pose[6], const int32_t src_dims[3], const float src_origin[3],
                   const float src_spacing[3], const float tgt_origin[3], const float tgt_spacing[3],
                   float mat_out[12], float a_out[3]) {
    if (!pose || !src_dims || !src_origin || !tgt_origin || !mat_out || !a_out)
        return fail(PF_EINVAL, "NULL argument");
    if (!spacing_ok(src_spacing) || !spacing_ok(tgt_spacing)) return fail(PF_EINVAL, "spacing outside (0, 1e6]");
    for (int d = 0; d < 6; ++d)
        if (!std::isfinite(pose[d])) return fail(PF_EINVAL, "pose is not finite");
    for (int d = 0; d < 3; ++d)
        if (!(std::fabs(pose[d]) <= kHalfPi)) return fail(PF_EINVAL, "rotation outside [-pi/2, pi/2]");
    const int32_t td[3] = {2, 2, 2};
    const Geometry g = make_geometry(src_dims, src_origin, src_spacing, td, tgt_origin, tgt_spacing);
    float *d = nullptr;
    CU(dev_malloc(&d, sizeof(float) * 18));
    cudaError_t e = cudaMemcpy(d, pose, sizeof(float) * 6, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_pose_matrix(d, g, d + 6, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(mat_out, d + 6, sizeof(float) * 12, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(PF_ECUDA, "pf_pose_matrix: %s", cudaGetErrorString(e));
    for (int i = 0; i < 3; ++i) a_out[i] = g.a[i];
    return PF_OK;
}

int pf_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    if (!ctr || !key || !out) return fail(PF_EINVAL, "NULL argument");
    uint32_t h[6] = {ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]};
    uint32_t *d = nullptr;
    CU(dev_malloc(&d, sizeof(uint32_t) * 10));
    cudaError_t e = cudaMemcpy(d, h, sizeof h, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_philox(d, d + 6, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 6, sizeof(uint32_t) * 4, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(PF_ECUDA, "pf_philox: %s", cudaGetErrorString(e));
    return PF_OK;
}

int warp_sequence(const uint8_t *const *frames_in, int32_t n_frames, const int32_t src_dims[3],
                  const float src_origin[3], const float src_spacing[3], uint8_t *const *frames_out,
                  const int32_t tgt_dims[3], const float tgt_origin[3], const float tgt_spacing[3],
                  const float pose[6], int32_t interp, void *cuda_stream) {
    NvtxRange nvtx("warp_sequence");
    if (!frames_in || !frames_out || !src_dims || !src_origin || !tgt_dims || !tgt_origin || !pose)
        return fail(PF_EINVAL, "NULL argument");
    if (n_frames < 0) return fail(PF_EINVAL, "n_frames < 0");
    if (interp != 0 && interp != 1) return fail(PF_EINVAL, "interp must be 0 or 1");
    for (int d = 0; d < 3; ++d) {
        if (src_dims[d] < 2 || src_dims[d] > kMaxDim || tgt_dims[d] < 1 || tgt_dims[d] > kMaxDim)
            return fail(PF_EINVAL, "dims out of range");
    }
    if (!finite3(src_origin) || !finite3(tgt_origin)) return fail(PF_EINVAL, "origin is not finite");
    for (int d = 0; d < 6; ++d)
        if (!std::isfinite(pose[d])) return fail(PF_EINVAL, "pose is not finite");
    for (int d = 0; d < 3; ++d)
        if (!(std::fabs(pose[d]) <= kHalfPi)) return fail(PF_EINVAL, "rotation outside [-pi/2, pi/2]");
    for (int32_t f = 0; f < n_frames; ++f)
        if (!frames_in[f] || !frames_out[f]) return fail(PF_EINVAL, "frame %d pointer is NULL", f);
    if (!spacing_ok(src_spacing) || !spacing_ok(tgt_spacing)) return fail(PF_EINVAL, "spacing outside (0, 1e6]");
    const Geometry g = make_geometry(src_dims, src_origin, src_spacing, tgt_dims, tgt_origin, tgt_spacing);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    for (int32_t f0 = 0; f0 < n_frames; f0 += WarpFrames::kMax) {
        WarpFrames wf;
        const int n = (n_frames - f0) < WarpFrames::kMax ? (n_frames - f0) : WarpFrames::kMax;
        for (int j = 0; j < WarpFrames::kMax; ++j) {
            wf.in[j] = j < n ? frames_in[f0 + j] : nullptr;
            wf.out[j] = j < n ? frames_out[f0 + j] : nullptr;
        }
        CU(launch_warp(wf, n, pose, g, interp, s));
    }
    return PF_OK;
}

}  // extern "C"

namespace pfreg {

// Measurement set-up of a context, for entry points defined in other files.
int ctx_measure_setup(pf_ctx *c, MeasureArgs *ma, bool *img, bool *mask, cudaStream_t *stream, int *device) {
    if (!c) return fail(PF_EINVAL, "ctx is NULL");
    *ma = c->MA;
    *img = c->img;
    *mask = c->mask;
    *stream = c->stream;
    *device = c->device;
    return PF_OK;
}

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

}  // namespace pfreg

// ---------------------------------------------------------------------------
// Batches of registrations stepped together.
// ---------------------------------------------------------------------------
struct pf_batch {
    std::vector<pf_ctx *> ctxs;        // in batch order: remaining iterations, descending
    std::vector<int32_t> remaining;    // iterations each member still has to run
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr, side[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    BatchReg *regs = nullptr;          // device table, batch order
    int32_t *lists = nullptr;          // three lists back to back: image, mask, combined
    long long *offs = nullptr;         // three item prefixes back to back (len + 1 each)
    long long *poffs = nullptr;        // particle prefix (n + 1)
    long long *poffs32 = nullptr;      // particle prefix, each member padded to whole warps
    int32_t *lptr[3] = {nullptr, nullptr, nullptr};
    long long *optr[3] = {nullptr, nullptr, nullptr};
    std::vector<int32_t> list_h[3];            // members of each list (batch positions)
    std::vector<int32_t> solo_h;               // members measured by their own launch (batch positions)
    std::vector<long long> offs_h[3], poffs_h, poffs32_h;
    std::map<int, cudaGraphExec_t> phase;      // graph per number of active members
    int ipw = kDefaultItemsPerWarp;            // tile shape of the measurement launches
    int max_tx[3] = {0, 0, 0};                 // longest target row of each list
    ~pf_batch() {
        for (auto &kv : phase) cudaGraphExecDestroy(kv.second);
        for (cudaStream_t s : {cap, side[0], side[1]})
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t e : {fork, join[0], join[1]})
            if (e) cudaEventDestroy(e);
        for (void *p : {(void *)regs, (void *)lists, (void *)offs, (void *)poffs, (void *)poffs32})
            if (p) cudaFree(p);
    }
};

namespace {

// Members of list k among the first `active` batch positions.
int list_prefix(const pf_batch *b, int k, int active) {
    const auto &L = b->list_h[k];
    return (int)(std::lower_bound(L.begin(), L.end(), active) - L.begin());
}

// Members with at least this many measurement work items (about four full
// waves of the single-registration kernel: 152 SMs x 3 CTAs x 8 warps x 8
// items each) are measured by their own launch inside the batch graph, with
// their own launch arguments, shared-memory mask bits and tile shape, spread
// over the graph's three streams; the concatenated launches serve the
// smaller members.  Timed on the mixed batches (16 members with 96-256
// voxels per axis; 64 members with 40-80): batched against sequential went
// from 0.89x to 1.01x and from 1.20x to 1.23x.  0: every member goes
// through the concatenated launches.
#ifndef PF_BATCH_SOLO_ITEMS
#define PF_BATCH_SOLO_ITEMS 120000
#endif
constexpr long long kSoloItems = PF_BATCH_SOLO_ITEMS;

int solo_prefix(const pf_batch *b, int active) {
    const auto &L = b->solo_h;
    return (int)(std::lower_bound(L.begin(), L.end(), active) - L.begin());
}

// The graph of one batch iteration with the first `active` members running:
// prediction of their particles, their measurements (three concurrent
// launches: image, mask and combined members), one update block each.  The
// grids cover exactly the active members' work.
int batch_phase_graph(pf_batch *b, int active, cudaGraphExec_t *out) {
    auto it = b->phase.find(active);
    if (it != b->phase.end()) {
        *out = it->second;
        return PF_OK;
    }
    int nl[3];
    for (int k = 0; k < 3; ++k) nl[k] = list_prefix(b, k, active);
    cudaGraph_t g = nullptr;
    g_capturing = true;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t es[12] = {cudaSuccess};
        es[0] = launch_predict_batch(b->regs, b->poffs, active, b->poffs_h[active], b->cap);
        es[1] = cudaEventRecord(b->fork, b->cap);
        es[2] = cudaStreamWaitEvent(b->side[0], b->fork, 0);
        es[3] = cudaStreamWaitEvent(b->side[1], b->fork, 0);
        es[4] = launch_measure_batch(b->regs, b->lptr[0], b->optr[0], nl[0], b->offs_h[0][nl[0]], true, false,
                                     b->ipw, b->max_tx[0], b->cap);
        es[5] = launch_measure_batch(b->regs, b->lptr[1], b->optr[1], nl[1], b->offs_h[1][nl[1]], false, true,
                                     b->ipw, b->max_tx[1], b->side[0]);
        es[6] = launch_measure_batch(b->regs, b->lptr[2], b->optr[2], nl[2], b->offs_h[2][nl[2]], true, true,
                                     b->ipw, b->max_tx[2], b->side[1]);
        // the large members' own launches, spread over the three streams
        const int ns = solo_prefix(b, active);
        for (int i = 0; i < ns && es[6] == cudaSuccess; ++i) {
            const pf_ctx *c = b->ctxs[b->solo_h[i]];
            es[6] = launch_measure(c->MA, c->img, c->mask, i % 3 == 0 ? b->cap : b->side[i % 3 - 1]);
        }
        es[7] = cudaEventRecord(b->join[0], b->side[0]);
        es[8] = cudaEventRecord(b->join[1], b->side[1]);
        es[9] = cudaStreamWaitEvent(b->cap, b->join[0], 0);
        es[10] = cudaStreamWaitEvent(b->cap, b->join[1], 0);
        es[11] = launch_finalise_batch(b->regs, b->poffs32, active, b->poffs32_h[active], b->cap);
        cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
        for (cudaError_t x : es)
            if (x != cudaSuccess && e == cudaSuccess) e = x;
        if (e == cudaSuccess) e = ee;
    }
    g_capturing = false;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(PF_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(PF_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
    b->phase[active] = x;
    *out = x;
    return PF_OK;
}

}  // namespace

extern "C" {

int pf_batch_create(pf_batch **out, pf_ctx *const *ctxs, int32_t n, const int32_t *n_iters) {
    if (!out) return fail(PF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || !n_iters || n < 1 || n > 65536) return fail(PF_EINVAL, "need 1..65536 contexts and counts");
    for (int32_t r = 0; r < n; ++r) {
        if (!ctxs[r]) return fail(PF_EINVAL, "context %d is NULL", r);
        if (n_iters[r] < 0) return fail(PF_EINVAL, "n_iters[%d] < 0", r);
        if (ctxs[r]->device != ctxs[0]->device) return fail(PF_EINVAL, "contexts are on different devices");
        if (ctxs[r]->stream != ctxs[0]->stream) return fail(PF_EINVAL, "contexts use different streams");
        for (int32_t q = 0; q < r; ++q)
            if (ctxs[q] == ctxs[r]) return fail(PF_EINVAL, "context %d appears twice", r);
    }
    // Batch order: remaining iterations descending, so the members still
    // running always form a prefix.
    std::vector<int32_t> rem(n);
    for (int32_t r = 0; r < n; ++r) {
        int32_t k = 0;
        int rc = pf_get_iteration(ctxs[r], &k);
        if (rc) return rc;
        rem[r] = n_iters[r] > k ? n_iters[r] - k : 0;
    }
    std::vector<int32_t> order(n);
    for (int32_t r = 0; r < n; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return rem[x] > rem[y]; });

    pf_batch *b = new (std::nothrow) pf_batch();
    if (!b) return fail(PF_ENOMEM, "host allocation failed");
    auto bail = [&](int code) {
        delete b;
        return code;
    };
#define BK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? PF_ENOMEM : PF_ECUDA, "%s: %s", #call, \
                             cudaGetErrorString(e_)));                                        \
    } while (0)
    b->stream = ctxs[0]->stream;
    std::vector<BatchReg> regs(n);
    b->poffs_h.assign(1, 0);
    b->poffs32_h.assign(1, 0);
    for (int k = 0; k < 3; ++k) b->offs_h[k].assign(1, 0);
    for (int32_t pos = 0; pos < n; ++pos) {
        pf_ctx *c = ctxs[order[pos]];
        b->ctxs.push_back(c);
        b->remaining.push_back(rem[order[pos]]);
        regs[pos].ma = c->MA;
        regs[pos].P = c->P;
        regs[pos].B = c->B;
        regs[pos].n_iters = n_iters[order[pos]];
        regs[pos].img = c->img;
        regs[pos].mask = c->mask;
        const int kind = (c->img && c->mask) ? 2 : (c->img ? 0 : 1);
        if (kSoloItems > 0 && measure_items(c->MA) >= kSoloItems) {
            b->solo_h.push_back(pos);
        } else {
            b->list_h[kind].push_back(pos);
            b->max_tx[kind] = std::max(b->max_tx[kind], (int)c->MA.g.td[0]);
            b->offs_h[kind].push_back(b->offs_h[kind].back() + measure_items(c->MA));
        }
        b->poffs_h.push_back(b->poffs_h.back() + c->P.N);
        b->poffs32_h.push_back(b->poffs32_h.back() + (c->P.N + 31) / 32 * 32);
    }
    BK(dev_malloc(&b->regs, sizeof(BatchReg) * n));
    BK(dev_malloc(&b->lists, sizeof(int32_t) * (size_t)n + 4));
    BK(dev_malloc(&b->offs, sizeof(long long) * (size_t)(n + 3)));
    BK(dev_malloc(&b->poffs, sizeof(long long) * (size_t)(n + 1)));
    BK(dev_malloc(&b->poffs32, sizeof(long long) * (size_t)(n + 1)));
    BK(cudaMemcpy(b->regs, regs.data(), sizeof(BatchReg) * n, cudaMemcpyHostToDevice));
    BK(cudaMemcpy(b->poffs, b->poffs_h.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
    BK(cudaMemcpy(b->poffs32, b->poffs32_h.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
    size_t lpos = 0, opos = 0;
    for (int k = 0; k < 3; ++k) {
        b->lptr[k] = b->lists + lpos;
        b->optr[k] = b->offs + opos;
        if (!b->list_h[k].empty())
            BK(cudaMemcpy(b->lptr[k], b->list_h[k].data(), sizeof(int32_t) * b->list_h[k].size(),
                          cudaMemcpyHostToDevice));
        BK(cudaMemcpy(b->optr[k], b->offs_h[k].data(), sizeof(long long) * b->offs_h[k].size(),
                      cudaMemcpyHostToDevice));
        lpos += b->list_h[k].size();
        opos += b->offs_h[k].size();
    }
    BK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    BK(cudaStreamCreateWithFlags(&b->side[0], cudaStreamNonBlocking));
    BK(cudaStreamCreateWithFlags(&b->side[1], cudaStreamNonBlocking));
    BK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    BK(cudaEventCreateWithFlags(&b->join[0], cudaEventDisableTiming));
    BK(cudaEventCreateWithFlags(&b->join[1], cudaEventDisableTiming));
#undef BK
    // Tile shape of the batch's measurement launches: tuned when every member
    // asked for it and none has run yet (the members' iteration-0 prediction
    // is repeatable, so the search can measure the real clouds).
    bool tune = true;
    for (int32_t r = 0; r < n; ++r) {
        int32_t k = 0;
        int rc = pf_get_iteration(ctxs[r], &k);
        if (rc) return bail(rc);
        tune = tune && ctxs[r]->cfg.autotune && k == 0;
    }
    if (tune) {
        for (pf_ctx *c : b->ctxs) {
            cudaError_t e = launch_predict(c->P, c->B, b->stream);
            if (e != cudaSuccess) return bail(fail(PF_ECUDA, "autotune: %s", cudaGetErrorString(e)));
        }
        int best = kDefaultItemsPerWarp;
        float ms = 0.0f;
        int rc = time_candidates(b->stream, [&](int ipw) {
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                const int nk = (int)b->list_h[k].size();
                e = launch_measure_batch(b->regs, b->lptr[k], b->optr[k], nk, b->offs_h[k][nk], k != 1, k != 0, ipw,
                                         b->max_tx[k], b->stream);
            }
            return e;
        }, &best, &ms);
        if (rc) return bail(rc);
        for (pf_ctx *c : b->ctxs) {
            cudaError_t e = cudaMemsetAsync(c->B.mom, 0, sizeof(unsigned long long) * kMomStride * (size_t)c->P.N,
                                            b->stream);
            if (e != cudaSuccess) return bail(fail(PF_ECUDA, "autotune: %s", cudaGetErrorString(e)));
        }
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bail(fail(PF_ECUDA, "autotune: %s", cudaGetErrorString(e)));
        b->ipw = best;
    }
    *out = b;
    return PF_OK;
}

int pf_batch_tile_shape(pf_batch *b, int32_t *items_per_warp) {
    if (!b || !items_per_warp) return fail(PF_EINVAL, "NULL argument");
    *items_per_warp = b->ipw;
    return PF_OK;
}

int pf_debug_alloc_limit(int64_t bytes) {
    if (bytes < 0) return fail(PF_EINVAL, "bytes < 0");
    g_alloc_limit.store(bytes);
    return PF_OK;
}

int pf_tile_shape(pf_ctx *c, int32_t *rows_per_item, int32_t *items_per_warp) {
    if (!c) return fail(PF_EINVAL, "ctx is NULL");
    if (rows_per_item) *rows_per_item = c->MA.rows_per_item;
    if (items_per_warp) *items_per_warp = c->MA.items_per_warp;
    return PF_OK;
}

int pf_batch_step(pf_batch *b, int32_t n_iters) {
    NvtxRange nvtx("pf_batch_step");
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    if (n_iters < 0) return fail(PF_EINVAL, "n_iters < 0");
    for (int32_t i = 0; i < n_iters; ++i) {
        int active = 0;
        while (active < (int)b->remaining.size() && b->remaining[active] > 0) ++active;
        if (active == 0) break;
        cudaGraphExec_t x = nullptr;
        int rc = batch_phase_graph(b, active, &x);
        if (rc) return rc;
        CU(cudaGraphLaunch(x, b->stream));
        int kernels = 4;   // prediction, scores, weights, update
        for (int k = 0; k < 3; ++k) kernels += list_prefix(b, k, active) > 0;
        kernels += solo_prefix(b, active);
        count_launches(kernels);
        for (int r = 0; r < active; ++r) --b->remaining[r];
    }
    return PF_OK;
}

int pf_batch_run(pf_batch *b) {
    if (!b) return fail(PF_EINVAL, "batch is NULL");
    return pf_batch_step(b, b->remaining.empty() ? 0 : b->remaining[0]);
}

int pf_batch_destroy(pf_batch *b) {
    if (!b) return PF_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    delete b;
    return PF_OK;
}

}  // extern "C"
