// Private to the library: the context record and the step orchestration shared by the
// public calls (api.cu) and the reverse sweep (adjoint.cu).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "../../include/lbmib.h"
#include "lbmib_kernels.cuh"

namespace lbmib {

constexpr size_t kAlign = 256;
constexpr int kMaxRing = 1024;

inline size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline size_t storage_bytes(lbmib_storage s) { return s == LBMIB_FP64 ? 8 : (s == LBMIB_FP32 ? 4 : 2); }

// Offsets of the context's buffers inside the caller's arena.
struct Layout {
    size_t pops[2], fib[2], mark, list[2], ctr, scratch;
    size_t X, Xm1, uv, Fint, Fext, U, L0, c0, s0, age, capid, mls, caps, obs, pts, pts_out;
    size_t Fpp, rep_box, rep_cellof, rep_count, rep_slot, u_in, rb, R0;
    int rep_buckets;
    size_t total;
    int pitch;
    long long plane;
};

}  // namespace lbmib

struct lbmib_ctx {
    int device = 0;  // the device that holds the arena
    lbmib_config cfg{};
    lbmib::Layout lay{};
    lbmib::Lat L{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    // Immersed-boundary kernels run on their own stream so that they overlap the lattice
    // update of the same or the next step (fork/join through these events).
    cudaStream_t ib_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_spread = nullptr, ev_patch = nullptr, ev_join = nullptr;
    int overlap = -1;   // 1 on, 0 off, -1 automatic (on while the capsules cannot fill the GPU)
    // the adjoint's third stream (a segment's recompute beside the previous segment's
    // reverse sweep) and the events of the reverse sweep's side-stream spread
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_adj[2]{};
    // capsule-capsule repulsion (Eq. 27); rep_rc = 0: off
    double rep_rc = 0.0, rep_coeff = 0.0;
    lbmib::RepGrid rep{};
    int sms = 0;        // multiprocessors of the device
    char* arena = nullptr;
    void* pops[2]{};
    double* fib[2]{};
    int* mark = nullptr;   // per node: the claim stamp of the last patch that forced it
    int* list[2]{};
    lbmib::DevCounters* ctr = nullptr;
    double* scratch = nullptr;
    lbmib::Nodes nd{};
    lbmib::CapsuleParams* d_caps = nullptr;
    double* obs = nullptr;
    double2* pts = nullptr;
    double* pts_out = nullptr;
    double* d_u_in = nullptr;   // inlet profile of an open channel (ny doubles)
    lbmib::OpenBC open{};       // open-channel data for the kernels that close the open columns
    std::vector<lbmib::CapsuleParams> caps;
    int max_n = 0;
    int nrigid = 0;           // rigid particles among the capsules
    double max_extent = 0.0;  // largest reference diameter of a capsule
    double max_arc_len = 0.0; // longest reference arc of the current split (slots included)
    int tile_cells = 256;     // per-CTA shared tile budget of the capsule kernels
    int arcs = 1;             // CTAs per capsule in the capsule kernels
    int arcs_opt = 0;         // requested arcs (0: automatic)
    int cur = 0;      // population buffer holding the latest post-collision state
    int cur_fib = 0;  // force buffer holding the last spread force
    long long steps = 0;
    long long launches = 0;
    // options
    bool use_graphs = true;
    bool timing = false;
    int graph_steps = 64;
    int lattice_variant = 256;
    bool fuse_ib = true;
    bool ib_fp64 = false;     // IB arithmetic in FP64 over single-precision storage
    // graphs keyed by (scheme, cur, cur_fib), with their steps and kernel launches
    cudaGraphExec_t graphs[2][2][2]{};
    int graph_len[2][2][2]{};
    long long graph_kernels[2][2][2]{};
    // timing
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    size_t ev_used = 0;
    double timed_ms = 0.0;
    long long timed_launches = 0;
    // the steps' patch and IB node-update kernels, timed from the lattice kernel's end
    // event (ev_pool[lat]) when every kernel of the step is on the lattice stream
    struct IbEvents {
        size_t lat;
        cudaEvent_t patch_end, ib_end;
    };
    std::vector<IbEvents> ev_ib;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_ib_free;
    double timed_patch_ms = 0.0, timed_ib_ms = 0.0;
    long long timed_ib_steps = 0;
    std::string err;
};

namespace lbmib {

lbmib_status fail(lbmib_ctx* c, lbmib_status s, const std::string& msg);
lbmib_status cuda_fail(lbmib_ctx* c, cudaError_t e, const char* where);

#define LBMIB_CUDA(ctx, call)                                              \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::lbmib::cuda_fail((ctx), e_, #call); \
    } while (0)

// Destroy the captured step graphs (after the buffers they name change role).
void drop_graphs(lbmib_ctx* c);

// Enqueue one coupled step on stream s: populations c->pops[cur] -> c->pops[1 - cur],
// last spread force c->fib[cur_fib]; advances (cur, cur_fib). With overlap on, the
// immersed-boundary kernels go to c->ib_stream: a sequence of steps must be bracketed
// by fork_ib() and join_ib() on s.
bool enqueue_step(lbmib_ctx* c, lbmib_scheme scheme, int& cur, int& cur_fib, cudaStream_t s, bool timed,
                  bool spread_done = false, bool fuse_next = false);
void fork_ib(lbmib_ctx* c, cudaStream_t s);
void join_ib(lbmib_ctx* c, cudaStream_t s);
// Whether the immersed-boundary kernels run on their own stream, and the stream they
// run on when a step sequence is enqueued on s.
bool overlapped(const lbmib_ctx* c);
inline cudaStream_t ib_stream_of(const lbmib_ctx* c, cudaStream_t s) { return overlapped(c) ? c->ib_stream : s; }

// Synchronise the context stream and translate the sticky device status.
lbmib_status device_status(lbmib_ctx* c);

template <typename F>
void by_storage(lbmib_storage st, F&& f) {
    if (st == LBMIB_FP64) f(double{});
    else if (st == LBMIB_FP32) f(float{});
    else f(__half{});
}

}  // namespace lbmib
