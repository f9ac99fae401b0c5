/* Lockstep emulation of one 32-lane warp on the host, for tests that run
 * warp-synchronous device code (shuffles, ballots, warp reductions) on the
 * CPU.  The 32 lanes are user-level contexts on one host thread, switched
 * round robin (ucontext): at every warp-level operation each lane posts its
 * value and passes control to the next lane; when the round comes back, all
 * 32 have posted, each reads what it needs, and a second round keeps any
 * lane from overwriting a slot before the others have read it.  Valid for
 * code whose warp operations are warp-uniform with the full mask, as the
 * measurement kernel's are.  host_warp::run(body) runs body(lane) on all
 * lanes.  Include this before anything that includes
 * tests/host_shim/cuda_runtime.h.  Test infrastructure only. */
#pragma once
#define PF_HOST_WARP_EMULATION 1
#include <ucontext.h>

#include <cstdint>
#include <cstring>
#include <functional>
#include <vector>

namespace host_warp {
inline ucontext_t main_ctx, lane_ctx[32];
inline int lane = 0;       // the lane running now
inline int finished = 0;   // lanes whose body has returned
inline uint64_t slot[32];
inline std::function<void(int)> body;

// hand control to the next lane; returns when the round comes back
inline void pass() {
    const int cur = lane, next = (cur + 1) & 31;
    lane = next;
    swapcontext(&lane_ctx[cur], &lane_ctx[next]);
    lane = cur;
}
inline void lane_main(int l) {
    body(l);
    if (++finished < 32) {   // the others are parked right after their last round
        lane = (l + 1) & 31;
        setcontext(&lane_ctx[lane]);
    }
    // the last lane returns to the caller through uc_link
}
inline void run(std::function<void(int)> f) {
    static std::vector<char> stacks((size_t)32 << 18);   // 256 KiB per lane
    body = std::move(f);
    finished = 0;
    for (int l = 0; l < 32; ++l) {
        getcontext(&lane_ctx[l]);
        lane_ctx[l].uc_stack.ss_sp = stacks.data() + ((size_t)l << 18);
        lane_ctx[l].uc_stack.ss_size = (size_t)1 << 18;
        lane_ctx[l].uc_link = &main_ctx;
        makecontext(&lane_ctx[l], (void (*)())lane_main, 1, l);
    }
    lane = 0;
    swapcontext(&main_ctx, &lane_ctx[0]);
}

// every lane posts v; returns what lane src posted
template <class T>
T exchange(T v, int src) {
    static_assert(sizeof(T) <= 8, "one slot per lane");
    uint64_t w = 0;
    std::memcpy(&w, &v, sizeof v);
    slot[lane] = w;
    pass();
    T r;
    std::memcpy(&r, &slot[src & 31], sizeof r);
    pass();
    return r;
}
}  // namespace host_warp

template <class T>
inline T __shfl_sync(unsigned, T v, int src) { return host_warp::exchange(v, src); }
inline unsigned long long __shfl_xor_sync(unsigned, unsigned long long v, int o) {
    return host_warp::exchange(v, host_warp::lane ^ o);
}
inline unsigned __ballot_sync(unsigned, int pred) {
    host_warp::slot[host_warp::lane] = pred ? 1u : 0u;
    host_warp::pass();
    unsigned m = 0;
    for (int l = 0; l < 32; ++l) m |= (unsigned)(host_warp::slot[l] & 1u) << l;
    host_warp::pass();
    return m;
}
inline unsigned __reduce_add_sync(unsigned, unsigned v) {
    host_warp::slot[host_warp::lane] = v;
    host_warp::pass();
    unsigned s = 0;
    for (int l = 0; l < 32; ++l) s += (unsigned)host_warp::slot[l];
    host_warp::pass();
    return s;
}
inline void __syncwarp() { host_warp::pass(); }
inline int __ffs(unsigned x) { return __builtin_ffs((int)x); }
// one host thread runs every lane, so a plain read-modify-write is atomic
inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) {
    const unsigned long long old = *p;
    *p = old + v;
    return old;
}
