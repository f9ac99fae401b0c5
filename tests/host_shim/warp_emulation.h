/* Lockstep emulation of one thread block on the host, for tests that run
 * warp-synchronous or block-synchronous device code (shuffles, ballots,
 * warp reductions, __syncthreads, shared memory) on the CPU.  Every thread
 * of the block is a user-level context on one host thread (ucontext), and
 * control passes round robin:
 *   a warp-level operation: each lane posts its value and hands control to
 *     the next lane of its warp; when the round comes back all 32 have
 *     posted, each reads what it needs, and a second round keeps any lane
 *     from overwriting a slot before the others have read it;
 *   __syncthreads: each thread hands control to the next thread of the block
 *     (warp-major), so when it resumes every thread has arrived.
 * Shared memory is the block's static storage (__shared__ is `static`), which
 * all contexts see.  Valid for code whose warp operations are uniform over
 * the warp's live lanes and whose barriers are uniform over the block's live
 * threads (a thread that has returned takes part in neither), as the
 * filter's kernels are.  host_warp::run(n, body) runs body(tid) on n threads
 * (a multiple of 32).  Include this before anything that includes
 * tests/host_shim/cuda_runtime.h.  Test infrastructure only. */
#pragma once
#define PF_HOST_WARP_EMULATION 1
#include <ucontext.h>

#include <cstdint>
#include <cstring>
#include <functional>
#include <vector>

namespace host_warp {
constexpr int kMaxThreads = 1024;
constexpr size_t kStack = (size_t)1 << 16;   // 64 KiB per thread
inline ucontext_t main_ctx, ctx[kMaxThreads];
inline int tid = 0;        // the thread running now
inline int nthreads = 32;
inline int finished = 0;   // threads whose body has returned
inline bool done[kMaxThreads];
inline uint64_t slot[kMaxThreads];
inline std::function<void(int)> body;

inline void switch_to(int next) {
    const int cur = tid;
    tid = next;
    swapcontext(&ctx[cur], &ctx[next]);
    tid = cur;
}
// hand control to the next live lane of this warp / the next live thread of
// the block (threads that have returned take no part, as on the device)
inline void pass_warp() {
    int next = (tid & ~31) | ((tid + 1) & 31);
    while (done[next]) next = (next & ~31) | ((next + 1) & 31);
    if (next != tid) switch_to(next);
}
inline void pass_block() {
    int next = (tid + 1) % nthreads;
    while (done[next]) next = (next + 1) % nthreads;
    if (next != tid) switch_to(next);
}

inline void thread_main(int t) {
    body(t);
    done[t] = true;
    if (++finished < nthreads) {   // the others are parked after their last rendezvous
        int next = (t + 1) % nthreads;
        while (done[next]) next = (next + 1) % nthreads;
        tid = next;
        setcontext(&ctx[next]);
    }
    // the last thread returns to the caller through uc_link
}
inline void run(int n, std::function<void(int)> f) {
    static std::vector<char> stacks((size_t)kMaxThreads * kStack);
    body = std::move(f);
    nthreads = n;
    finished = 0;
    for (int t = 0; t < n; ++t) {
        done[t] = false;
        getcontext(&ctx[t]);
        ctx[t].uc_stack.ss_sp = stacks.data() + (size_t)t * kStack;
        ctx[t].uc_stack.ss_size = kStack;
        ctx[t].uc_link = &main_ctx;
        makecontext(&ctx[t], (void (*)())thread_main, 1, t);
    }
    tid = 0;
    swapcontext(&main_ctx, &ctx[0]);
}
inline void run(std::function<void(int)> f) { run(32, std::move(f)); }

// every lane of the warp posts v; returns what lane src of the warp posted
template <class T>
T exchange(T v, int src) {
    static_assert(sizeof(T) <= 8, "one slot per thread");
    uint64_t w = 0;
    std::memcpy(&w, &v, sizeof v);
    slot[tid] = w;
    pass_warp();
    T r;
    std::memcpy(&r, &slot[(tid & ~31) | (src & 31)], sizeof r);
    pass_warp();
    return r;
}
}  // namespace host_warp

template <class T>
inline T __shfl_sync(unsigned, T v, int src) { return host_warp::exchange(v, src); }
template <class T>
inline T __shfl_xor_sync(unsigned, T v, int o) { return host_warp::exchange(v, (host_warp::tid & 31) ^ o); }
template <class T>
inline T __shfl_up_sync(unsigned, T v, unsigned d) {
    const int l = host_warp::tid & 31;
    const T r = host_warp::exchange(v, l >= (int)d ? l - (int)d : l);
    return r;
}
inline unsigned __ballot_sync(unsigned, int pred) {
    const int base = host_warp::tid & ~31;
    host_warp::slot[host_warp::tid] = pred ? 1u : 0u;
    host_warp::pass_warp();
    unsigned m = 0;
    for (int l = 0; l < 32; ++l) m |= (unsigned)(host_warp::slot[base + l] & 1u) << l;
    host_warp::pass_warp();
    return m;
}
inline unsigned __reduce_add_sync(unsigned, unsigned v) {
    const int base = host_warp::tid & ~31;
    host_warp::slot[host_warp::tid] = v;
    host_warp::pass_warp();
    unsigned s = 0;
    for (int l = 0; l < 32; ++l) s += (unsigned)host_warp::slot[base + l];
    host_warp::pass_warp();
    return s;
}
inline void __syncwarp(unsigned = 0xffffffffu) { host_warp::pass_warp(); }
inline void __syncthreads() { host_warp::pass_block(); }
inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
// one host thread runs every context, so a plain read-modify-write is atomic
inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) {
    const unsigned long long old = *p;
    *p = old + v;
    return old;
}
inline unsigned long long atomicMax(unsigned long long *p, unsigned long long v) {
    const unsigned long long old = *p;
    if (v > old) *p = v;
    return old;
}
