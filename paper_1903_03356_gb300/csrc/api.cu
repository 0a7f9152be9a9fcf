// C ABI of the LBM-IB library (declared in include/lbmib.h): context, arena layout,
// step orchestration with CUDA-graph replay, read-back and checkpoints.
//
// One coupled step (Coclite et al., arXiv:1903.03356) is enqueued as
//   Dynamic   (Section 2.3.2): force+spread (steps 1-3) | collide-stream (4-6) |
//             forced-node patch | per-capsule update (7-8)
//   Kinematic (Section 2.4):   force+spread (i-iii) | collide-stream (iv-vi) |
//             forced-node patch | advance (vii-viii)
// The collide-stream kernel applies only the uniform body force; the patch redoes the
// collision of the few nodes in the support of a marker with the spread force, so the
// hot loop stays at 18 population transfers per lattice update. Two force buffers
// alternate: a step spreads into one while interpolation reads the last spread force
// from the other; the patch of a step clears the older buffer at its touched cells.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ctx.cuh"

using namespace lbmib;
namespace {

bool valid_config(const lbmib_config* c) {
    return c && c->nx >= 3 && c->ny >= 3 && c->tau > 0.5 && c->max_capsules >= 0 && c->max_nodes >= 0 &&
           (c->storage == LBMIB_FP64 || c->storage == LBMIB_FP32 || c->storage == LBMIB_FP16) &&
           (long long)c->nx * c->ny < (1LL << 31) && c->max_nodes <= (1 << 26);
}

Layout make_layout(const lbmib_config* c) {
    Layout L{};
    const size_t s = storage_bytes(c->storage);
    L.pitch = (int)up((size_t)c->nx, 128 / s);
    L.plane = (long long)c->ny * L.pitch;
    const size_t N = (size_t)c->nx * c->ny;
    const size_t M = (size_t)(c->max_nodes > 0 ? c->max_nodes : 1);
    const size_t K = (size_t)(c->max_capsules > 0 ? c->max_capsules : 1);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = up(o + bytes, kAlign); return r; };
    L.pops[0] = take(9 * (size_t)L.plane * s);
    L.pops[1] = take(9 * (size_t)L.plane * s);
    L.fib[0] = take(2 * N * sizeof(double));
    L.fib[1] = take(2 * N * sizeof(double));
    L.mark = take(N * sizeof(int));
    L.list[0] = take(9 * M * sizeof(int));
    L.list[1] = take(9 * M * sizeof(int));
    L.ctr = take(sizeof(DevCounters));
    L.scratch = take(3 * N * sizeof(double));
    L.X = take(M * sizeof(double2));
    L.Xm1 = take(M * sizeof(double2));
    L.uv = take(M * sizeof(double2));
    L.Fint = take(M * sizeof(double2));
    L.Fext = take(M * sizeof(double2));
    L.U = take(M * sizeof(double2));
    L.L0 = take(M * sizeof(double));
    L.c0 = take(M * sizeof(double));
    L.s0 = take(M * sizeof(double));
    L.age = take(M * sizeof(int));
    L.capid = take(M * sizeof(int));
    L.mls = take(M * sizeof(MlsW<double>));
    L.caps = take(K * sizeof(CapsuleParams));
    L.obs = take(8 * K * sizeof(double));
    L.Fpp = take(M * sizeof(double2));
    L.rep_buckets = 64;
    while (L.rep_buckets < 4 * (int)K) L.rep_buckets *= 2;
    L.rep_box = take(4 * K * sizeof(double));
    L.rep_cellof = take(K * sizeof(int));
    L.rep_count = take((size_t)L.rep_buckets * sizeof(int));
    L.rep_slot = take((size_t)L.rep_buckets * kRepSlots * sizeof(int));
    L.pts = take(M * sizeof(double2));
    L.pts_out = take(8 * M * sizeof(double));
    L.u_in = take((size_t)c->ny * sizeof(double));
    L.rb = take(K * sizeof(RigidBody));
    L.R0 = take(M * sizeof(double2));
    L.total = o;
    return L;
}

}  // namespace

namespace lbmib {

lbmib_status fail(lbmib_ctx* c, lbmib_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

lbmib_status cuda_fail(lbmib_ctx* c, cudaError_t e, const char* where) {
    return fail(c, LBMIB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}



void drop_graphs(lbmib_ctx* c) {
    for (auto& a : c->graphs)
        for (auto& b : a)
            for (auto& g : b)
                if (g) {
                    cudaGraphExecDestroy(g);
                    g = nullptr;
                }
}

// Stream schedule of one step (FS force+spread, CS collide-stream, P patch, U update):
//   ib stream:      FS(n) ----------+                 +--> U(n) --> FS(n+1) ...
//   lattice stream: CS(n) ------- wait --> P(n) --+---+--> CS(n+1) ...
// CS reads only the populations and the uniform force, so it does not wait for FS; P
// needs both. CS(n+1) needs the patched populations only, so it runs beside U(n) and
// FS(n+1), which read those populations and write vertices, lists and the other force
// buffer. The lattice kernel is HBM-bound and the IB kernels FP64- and latency-bound,
// so the two can share the GPU. Measured on GB300: with few capsules (one CTA each,
// most SMs idle during the IB kernels) the step time drops by a third; with enough
// capsules to fill the GPU the IB blocks take registers and warp slots from the lattice
// kernel, which slows by what the overlap saves. Hence the automatic setting: overlap
// while the capsules number fewer than two per SM.
bool overlapped(const lbmib_ctx* c) {
    if (c->caps.empty() || c->overlap == 0) return false;
    return c->overlap == 1 || (int)c->caps.size() < 2 * (c->sms > 0 ? c->sms : 1);
}

void fork_ib(lbmib_ctx* c, cudaStream_t s) {
    if (!overlapped(c)) return;
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(c->ib_stream, c->ev_fork, 0);
}

void join_ib(lbmib_ctx* c, cudaStream_t s) {
    if (!overlapped(c)) return;
    cudaEventRecord(c->ev_join, c->ib_stream);
    cudaStreamWaitEvent(s, c->ev_join, 0);
}

// Calls f with a value of the storage type the immersed-boundary kernels are instantiated
// on: the storage itself, or with LBMIB_OPT_IB_FP64 over single-precision storage its
// widening view (gathers in storage precision, the IB arithmetic in FP64).
template <typename F>
void with_ib_storage(const lbmib_ctx* c, F&& f) {
    switch (c->cfg.storage) {
        case LBMIB_FP64: f(double{}); break;
        case LBMIB_FP32:
            if (c->ib_fp64) f(f32w{});
            else f(float{});
            break;
        default:
            if (c->ib_fp64) f(f16w{});
            else f(__half{});
    }
}

// Whether the Dynamic node update of a step may also do the force and spread of the next
// (k_dyn_update_spread): one CTA per capsule and no rigid particles.
bool fusable(const lbmib_ctx* c) { return c->fuse_ib && c->arcs == 1 && c->nrigid == 0 && !c->caps.empty(); }

// Enqueue one coupled step on stream s, advancing (cur, cur_fib). `spread_done`: the
// previous step's update already did this step's force and spread; `fuse_next`: another
// step of the same scheme follows in this run, so the update may do its force and
// spread. Returns whether it did.
bool enqueue_step(lbmib_ctx* c, lbmib_scheme scheme, int& cur, int& cur_fib, cudaStream_t s_lat, bool timed,
                  bool spread_done, bool fuse_next) {
    const Lat& L = c->L;
    const int ncaps = (int)c->caps.size();
    const bool ov = overlapped(c);
    cudaStream_t s = ov ? c->ib_stream : s_lat;   // stream of the immersed-boundary kernels
    const void* src = c->pops[cur];
    void* dst = c->pops[1 - cur];
    const int fc = 1 - cur_fib;  // buffer spread into this step
    const int fp = cur_fib;      // last spread force
    unsigned* status = &c->ctr->status;
    const int list_cap = 9 * (c->cfg.max_nodes > 0 ? c->cfg.max_nodes : 1);
    Spread sp{c->fib[fc], c->list[fc], &c->ctr->count[fc], list_cap, status};
    const lbmib_storage st = c->cfg.storage;
    if (ncaps > 1 && c->rep_rc > 0.0) {
        launch_repulsion(L, c->nd, ncaps, c->max_n, c->arcs, c->rep, status, s);
        c->launches += 2;
    }
    if (ncaps > 0 && !spread_done) {
        if (scheme == LBMIB_DYNAMIC) {
            with_ib_storage(c, [&](auto v) {
                launch_dyn_force_spread<decltype(v)>(src, L, c->nd, ncaps, c->max_n, c->arcs, c->tile_cells,
                                                     c->nrigid > 0, sp, status, s);
            });
        } else {
            launch_kin_force_spread(L, c->nd, ncaps, c->max_n, c->arcs, c->tile_cells, sp, status,
                                    st == LBMIB_FP64 || c->ib_fp64, s);
        }
        c->launches++;
        if (ov) cudaEventRecord(c->ev_spread, s);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed) {
        if (c->ev_used == c->ev_pool.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            c->ev_pool.push_back({a, b});
        }
        e0 = c->ev_pool[c->ev_used].first;
        e1 = c->ev_pool[c->ev_used].second;
        c->ev_used++;
        cudaEventRecord(e0, s_lat);
    }
    if (st == LBMIB_FP64) launch_collide_stream<double>(src, dst, L, status, c->lattice_variant, s_lat);
    else if (st == LBMIB_FP32) launch_collide_stream<float>(src, dst, L, status, c->lattice_variant, s_lat);
    else launch_collide_stream<__half>(src, dst, L, status, c->lattice_variant, s_lat);
    c->launches++;
    if (timed) cudaEventRecord(e1, s_lat);
    if (L.inflow) {   // open channel: the inlet and outlet columns, over the lattice kernel's output
        if (st == LBMIB_FP64) launch_open_columns<double>(src, dst, L, c->open, status, s_lat);
        else if (st == LBMIB_FP32) launch_open_columns<float>(src, dst, L, c->open, status, s_lat);
        else launch_open_columns<__half>(src, dst, L, c->open, status, s_lat);
        c->launches++;
    }
    if (ncaps > 0) {
        const int cap = list_cap;
        if (ov) cudaStreamWaitEvent(s_lat, c->ev_spread, 0);
        if (st == LBMIB_FP64)
            launch_patch<double>(dst, L, c->fib[fc], c->list[fc], c->fib[fp], c->list[fp], c->mark, c->ctr, fc, cap,
                                   c->nd.count, s_lat);
        else if (st == LBMIB_FP32)
            launch_patch<float>(dst, L, c->fib[fc], c->list[fc], c->fib[fp], c->list[fp], c->mark, c->ctr, fc, cap,
                                   c->nd.count, s_lat);
        else
            launch_patch<__half>(dst, L, c->fib[fc], c->list[fc], c->fib[fp], c->list[fp], c->mark, c->ctr, fc, cap,
                                   c->nd.count, s_lat);
        if (ov) {
            cudaEventRecord(c->ev_patch, s_lat);
            cudaStreamWaitEvent(s, c->ev_patch, 0);
        }
        // patch and IB node-update times (one stream only: with overlap the IB kernels run
        // beside the next lattice update)
        const bool time_ib = timed && !ov && !L.inflow;
        cudaEvent_t ep = nullptr, ei = nullptr;
        if (time_ib) {
            if (c->ev_ib_free.empty()) {
                cudaEvent_t a, b;
                cudaEventCreate(&a);
                cudaEventCreate(&b);
                c->ev_ib_free.push_back({a, b});
            }
            ep = c->ev_ib_free.back().first;
            ei = c->ev_ib_free.back().second;
            c->ev_ib_free.pop_back();
            c->ev_ib.push_back({c->ev_used - 1, ep, ei});
            cudaEventRecord(ep, s_lat);
        }
        int* reset = &c->ctr->count[fp];
        if (scheme == LBMIB_DYNAMIC && fuse_next && fusable(c)) {
            // the next step spreads into the buffer and list this step's patch has just
            // cleared and read: reset their counter first (the fused kernel appends to it)
            cudaMemsetAsync(reset, 0, sizeof(int), s);
            const Spread next{c->fib[fp], c->list[fp], reset, list_cap, status};
            with_ib_storage(c, [&](auto v) {
                launch_dyn_update_spread<decltype(v)>(dst, L, c->nd, ncaps, c->max_n, c->tile_cells, next,
                                                      status, s);
            });
            if (ov) cudaEventRecord(c->ev_spread, s);
            if (time_ib) cudaEventRecord(ei, s);
            c->launches += 2;
            cur_fib = fc;
            cur = 1 - cur;
            return true;
        }
        if (scheme == LBMIB_KINEMATIC && fuse_next && fusable(c) && !(ncaps > 1 && c->rep_rc > 0.0)) {
            // as above; the Kinematic spread also needs the repulsion at X^{n+1}, which the
            // next step computes first: fused only without repulsion
            cudaMemsetAsync(reset, 0, sizeof(int), s);
            const Spread next{c->fib[fp], c->list[fp], reset, list_cap, status};
            with_ib_storage(c, [&](auto v) {
                launch_kin_advance_spread<decltype(v)>(dst, L, c->fib[fc], c->nd, ncaps, c->max_n, c->tile_cells,
                                                       next, status, s);
            });
            if (ov) cudaEventRecord(c->ev_spread, s);
            if (time_ib) cudaEventRecord(ei, s);
            c->launches += 2;
            cur_fib = fc;
            cur = 1 - cur;
            return true;
        }
        if (scheme == LBMIB_DYNAMIC) {
            with_ib_storage(c, [&](auto v) {
                launch_dyn_update<decltype(v)>(dst, L, c->nd, ncaps, c->max_n, c->arcs, c->tile_cells,
                                               c->nrigid > 0, reset, status, s);
            });
        } else {
            with_ib_storage(c, [&](auto v) {
                launch_kin_advance<decltype(v)>(dst, L, c->fib[fc], c->nd, ncaps, c->max_n, c->arcs, c->tile_cells,
                                                reset, status, s);
            });
        }
        if (time_ib) cudaEventRecord(ei, s);
        c->launches += 2;
        cur_fib = fc;
    }
    cur = 1 - cur;
    return false;
}

// Enqueue n steps of one scheme on stream s, fusing each Dynamic update with the next
// step's force and spread where fusable.
void enqueue_steps(lbmib_ctx* c, lbmib_scheme scheme, long long n, int& cur, int& cur_fib, cudaStream_t s, bool timed) {
    bool ahead = false;
    for (long long k = 0; k < n; k++) ahead = enqueue_step(c, scheme, cur, cur_fib, s, timed, ahead, k + 1 < n);
}

lbmib_status device_status(lbmib_ctx* c) {
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    unsigned st = 0;
    LBMIB_CUDA(c, cudaMemcpy(&st, &c->ctr->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st & kStatUnstable) return fail(c, LBMIB_ERR_UNSTABLE, "unstable lattice: |u| > 0.3 or NaN");
    if (st & kStatSupport) return fail(c, LBMIB_ERR_SUPPORT, "an MLS support or probe left the channel");
    if (st & kStatTimeout) return fail(c, LBMIB_ERR_TIMEOUT, "a bounded device wait gave up");
    if (st & kStatGrid)
        return fail(c, LBMIB_ERR_STATE, "repulsion neighbour grid: a capsule outgrew its cell or a bucket overflowed");
    if (st & (kStatList | kStatCell | kStatRing))
        return fail(c, LBMIB_ERR_STATE, "device bookkeeping check failed (status bits " + std::to_string(st) + ")");
    return LBMIB_OK;
}

}  // namespace lbmib

namespace {

// Arcs per capsule: one CTA per capsule while the capsules fill the multiprocessors;
// with fewer capsules, up to kMaxArcs CTAs per capsule (at least 16 vertices each) so
// that the capsule kernels still spread over the GPU (measured on a 128-vertex ring:
// 1, 2, 4, 8 arcs give 61, 49, 41, 39 us per Dynamic step). Then the tile budget for arcs of
// the longest reference arc (1.5 x for stretching), capped by the capsule diameter; a
// box that outgrows it takes the global path, with the same results.
void update_arcs(lbmib_ctx* c) {
    const int ncaps = (int)c->caps.size();
    int a = c->arcs_opt;
    if (a == 0) {
        const int sms = c->sms > 0 ? c->sms : 1;
        a = ncaps == 0 || ncaps >= sms ? 1 : std::min({kMaxArcs, sms / ncaps, (c->max_n + 15) / 16});
        a = std::max(a, 1);
    }
    auto arc_of = [a](const CapsuleParams& P) {
        return P.P0 * (double)((P.n + a - 1) / a + 2 * kHalo) / (double)P.n;
    };
    double arc = 0.0;
    if (a == c->arcs && !c->caps.empty()) arc = std::max(c->max_arc_len, arc_of(c->caps.back()));
    else
        for (const CapsuleParams& P : c->caps) arc = std::max(arc, arc_of(P));
    const int slots = arc_slots(std::max(c->max_n, 1), a);
    // a curve of length l fits a box of w + h <= sqrt(2) l, so a split arc's box is at
    // most l / sqrt(2) on a side on average: budget for that square (with 1.5 x l)
    const double reach = std::min(c->max_extent, 1.5 * arc);
    const int cells = tile_budget(slots, a > 1 ? reach / std::sqrt(2.0) : reach, a > 1);
    c->arcs = a;
    c->max_arc_len = arc;
    c->tile_cells = cells;
    set_capsule_smem_limits(slots, cells);
    drop_graphs(c);   // launch shapes may have changed
}


// Neighbour grid of the repulsion for the current capsules: coarse cells at least
// 1.5 x the largest reference extent plus the cut-off (room for deformation; the bin
// kernel flags a capsule that outgrows it), a whole number of cells per axis.
void update_rep_grid(lbmib_ctx* c) {
    RepGrid& g = c->rep;
    g.rc = c->rep_rc;
    g.coeff = c->rep_coeff;
    const double want = 1.5 * c->max_extent + c->rep_rc + 1.0;
    g.ncx = std::max(1, (int)std::floor(c->cfg.nx / want));
    g.ncy = std::max(1, (int)std::floor(c->cfg.ny / want));
    g.cellx = (double)c->cfg.nx / g.ncx;
    g.celly = (double)c->cfg.ny / g.ncy;
    c->nd.Fpp = c->rep_rc > 0.0 ? (double2*)(c->arena + c->lay.Fpp) : nullptr;
}

lbmib_status capture(lbmib_ctx* c, lbmib_scheme scheme, int cur, int cur_fib, int len, cudaGraphExec_t* out,
                     long long* kernels) {
    LBMIB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long launches = c->launches;
    fork_ib(c, c->cap_stream);
    enqueue_steps(c, scheme, len, cur, cur_fib, c->cap_stream, false);
    join_ib(c, c->cap_stream);
    *kernels = c->launches - launches;
    c->launches = launches;  // capture does not launch
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    return LBMIB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------
// Staging memory of lbmib_interpolate_noalloc: a file-scope device array, so that the
// call needs no allocation by anyone. Every device that loads the library holds it
// (1.25 MiB) until the process exits. In host code the name g_noalloc_interp is only a
// stand-in for the symbol; the device address comes from cudaGetSymbolAddress, taken
// once per device with that device current and cached in g_noalloc_addr.
// ---------------------------------------------------------------------------------
namespace {
constexpr int kNoallocMaxPoints = 16384;
constexpr int kNoallocMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_interp[kNoallocMaxPoints * 10];  // 2 in + 8 out per point
double* g_noalloc_addr[kNoallocMaxDevices] = {};
std::mutex g_noalloc_mu;
}  // namespace

extern "C" {

size_t lbmib_arena_bytes(const lbmib_config* cfg) {
    if (!valid_config(cfg)) return 0;
    return make_layout(cfg).total;
}

lbmib_status lbmib_create(const lbmib_config* cfg, void* d_arena, size_t arena_bytes, void* cuda_stream,
                          lbmib_ctx** out) {
    if (!out) return LBMIB_ERR_ARG;
    *out = nullptr;
    if (!valid_config(cfg)) return LBMIB_ERR_ARG;
    const Layout lay = make_layout(cfg);
    if (!d_arena || ((uintptr_t)d_arena % kAlign) != 0) return LBMIB_ERR_ARG;
    if (arena_bytes < lay.total) return LBMIB_ERR_OOM;
    lbmib_ctx* c = new lbmib_ctx();
    c->cfg = *cfg;
    {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, d_arena) == cudaSuccess && pa.type == cudaMemoryTypeDevice)
            c->device = pa.device;
        else
            cudaGetDevice(&c->device);
        cudaGetLastError();  // clear a non-sticky error from the attribute query
    }
    c->lay = lay;
    c->stream = (cudaStream_t)cuda_stream;
    c->arena = (char*)d_arena;
    char* a = c->arena;
    c->pops[0] = a + lay.pops[0];
    c->pops[1] = a + lay.pops[1];
    c->fib[0] = (double*)(a + lay.fib[0]);
    c->fib[1] = (double*)(a + lay.fib[1]);
    c->mark = (int*)(a + lay.mark);
    c->list[0] = (int*)(a + lay.list[0]);
    c->list[1] = (int*)(a + lay.list[1]);
    c->ctr = (DevCounters*)(a + lay.ctr);
    c->scratch = (double*)(a + lay.scratch);
    c->nd.X = (double2*)(a + lay.X);
    c->nd.Xm1 = (double2*)(a + lay.Xm1);
    c->nd.uv = (double2*)(a + lay.uv);
    c->nd.Fint = (double2*)(a + lay.Fint);
    c->nd.Fext = (double2*)(a + lay.Fext);
    c->nd.U = (double2*)(a + lay.U);
    c->nd.L0 = (double*)(a + lay.L0);
    c->nd.c0 = (double*)(a + lay.c0);
    c->nd.s0 = (double*)(a + lay.s0);
    c->nd.age = (int*)(a + lay.age);
    c->nd.capid = (int*)(a + lay.capid);
    c->nd.mls = a + lay.mls;
    c->nd.Fpp = nullptr;   // set while repulsion is on
    c->nd.rb = (RigidBody*)(a + lay.rb);
    c->nd.R0 = (double2*)(a + lay.R0);
    c->rep.count = (int*)(a + lay.rep_count);
    c->rep.slot = (int*)(a + lay.rep_slot);
    c->rep.cellof = (int*)(a + lay.rep_cellof);
    c->rep.box = (double*)(a + lay.rep_box);
    c->rep.nbuckets = lay.rep_buckets;
    c->d_caps = (CapsuleParams*)(a + lay.caps);
    c->nd.caps = c->d_caps;
    c->nd.count = 0;
    c->obs = (double*)(a + lay.obs);
    c->pts = (double2*)(a + lay.pts);
    c->pts_out = (double*)(a + lay.pts_out);
    c->d_u_in = (double*)(a + lay.u_in);

    Lat& L = c->L;
    L.nx = cfg->nx;
    L.ny = cfg->ny;
    L.pitch = lay.pitch;
    L.plane = lay.plane;
    L.walls = cfg->walls ? 1 : 0;
    L.tau = cfg->tau;
    L.omega = 1.0 / cfg->tau;
    L.ub = cfg->walls ? cfg->u_bottom : 0.0;
    L.ut = cfg->walls ? cfg->u_top : 0.0;
    L.gx = cfg->gx;
    L.gy = cfg->gy;
    L.scale = cfg->storage == LBMIB_FP16 ? 1024.0f : 1.0f;
    L.inv_scale = 1.0f / L.scale;
    L.nu = (cfg->tau - 0.5) / 3.0;
    // lattice launch shape measured fastest on GB300: 128-thread blocks, and for the
    // single-precision storages a 64-register cap (eight resident blocks per SM)
    c->lattice_variant = cfg->storage == LBMIB_FP64 ? 0x80 : (0x80 | (1 << 18));
    if (cfg->storage == LBMIB_FP16) c->lattice_variant |= 1 << 19;   // packed 16-byte FP16 kernel
    L.gxf = (float)L.gx;
    L.gyf = (float)L.gy;
    L.omegaf = (float)L.omega;
    L.ubf = (float)L.ub;
    L.utf = (float)L.ut;

    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->ib_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&c->ev_fork, &c->ev_spread, &c->ev_patch, &c->ev_join, &c->ev_adj[0], &c->ev_adj[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lbmib_destroy(c);
        return LBMIB_ERR_CUDA;
    }
    set_capsule_smem_limits(1, c->tile_cells);
    const size_t N = (size_t)cfg->nx * cfg->ny;
    e = cudaMemsetAsync(c->fib[0], 0, 2 * N * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fib[1], 0, 2 * N * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->mark, 0, N * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), c->stream);
    if (e != cudaSuccess) {
        lbmib_destroy(c);
        return LBMIB_ERR_CUDA;
    }
    by_storage(cfg->storage, [&](auto tag) {
        using S = decltype(tag);
        launch_init<S>(c->pops[0], c->L, nullptr, nullptr, nullptr, c->stream);
    });
    c->launches++;
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbmib_destroy(c);
        return LBMIB_ERR_CUDA;
    }
    *out = c;
    return LBMIB_OK;
}

void lbmib_destroy(lbmib_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (auto& p : c->ev_pool) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    for (const auto& e : c->ev_ib) c->ev_ib_free.push_back({e.patch_end, e.ib_end});
    for (auto& p : c->ev_ib_free) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaStream_t* q : {&c->ib_stream, &c->aux_stream})
        if (*q) {
            cudaStreamSynchronize(*q);
            cudaStreamDestroy(*q);
        }
    for (cudaEvent_t ev : {c->ev_fork, c->ev_spread, c->ev_patch, c->ev_join, c->ev_adj[0], c->ev_adj[1]})
        if (ev) cudaEventDestroy(ev);
    delete c;
}

const char* lbmib_last_error(const lbmib_ctx* c) { return c ? c->err.c_str() : "null context"; }

lbmib_status lbmib_init_fields(lbmib_ctx* c, const double* rho, const double* ux, const double* uy) {
    if (!c) return LBMIB_ERR_ARG;
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    double* d[3] = {c->scratch, c->scratch + N, c->scratch + 2 * N};
    const double* h[3] = {rho, ux, uy};
    for (int k = 0; k < 3; k++)
        if (h[k]) LBMIB_CUDA(c, cudaMemcpyAsync(d[k], h[k], N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    by_storage(c->cfg.storage, [&](auto tag) {
        using S = decltype(tag);
        launch_init<S>(c->pops[c->cur], c->L, rho ? d[0] : nullptr, ux ? d[1] : nullptr, uy ? d[2] : nullptr,
                       c->stream);
    });
    c->launches++;
    LBMIB_CUDA(c, cudaMemsetAsync(c->fib[0], 0, 2 * N * sizeof(double), c->stream));
    LBMIB_CUDA(c, cudaMemsetAsync(c->fib[1], 0, 2 * N * sizeof(double), c->stream));
    LBMIB_CUDA(c, cudaMemsetAsync(c->ctr->count, 0, sizeof(c->ctr->count), c->stream));
    LBMIB_CUDA(c, cudaGetLastError());
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBMIB_OK;
}

static void ring_reference(const double* xy, int n, std::vector<double>& L0, std::vector<double>& c0,
                           std::vector<double>& s0, double& A0, double& P0) {
    L0.resize(n);
    c0.resize(n);
    s0.resize(n);
    double a2 = 0.0, per = 0.0;
    for (int v = 0; v < n; v++) {
        const int r = (v + 1) % n, l = (v + n - 1) % n;
        const double dx = xy[2 * r] - xy[2 * v], dy = xy[2 * r + 1] - xy[2 * v + 1];
        L0[v] = std::sqrt(dx * dx + dy * dy);
        per += L0[v];
        const double ax = xy[2 * v] - xy[2 * l], ay = xy[2 * v + 1] - xy[2 * l + 1];
        const double nrm = std::sqrt((ax * ax + ay * ay) * (dx * dx + dy * dy));
        c0[v] = (ax * dx + ay * dy) / nrm;  // cos(theta_0)
        s0[v] = (ax * dy - ay * dx) / nrm;  // sin(theta_0)
        a2 += (xy[2 * v] - xy[0]) * (xy[2 * r + 1] - xy[1]) - (xy[2 * r] - xy[0]) * (xy[2 * v + 1] - xy[1]);
    }
    A0 = 0.5 * a2;
    P0 = per;
}

lbmib_status lbmib_add_capsule(lbmib_ctx* c, const double* xy, int n, double ks, double kb, double ka,
                               double node_mass, int* id_out) {
    if (!c) return LBMIB_ERR_ARG;
    if (!xy || n < 3 || n > kMaxRing || !(node_mass > 0.0)) return fail(c, LBMIB_ERR_ARG, "bad capsule arguments");
    if ((int)c->caps.size() >= c->cfg.max_capsules || c->nd.count + n > c->cfg.max_nodes)
        return fail(c, LBMIB_ERR_OOM, "capsule capacity exceeded");
    std::vector<double> L0, c0, s0;
    double A0, P0;
    ring_reference(xy, n, L0, c0, s0, A0, P0);
    if (!(A0 > 0.0)) return fail(c, LBMIB_ERR_ARG, "capsule ring must be counter-clockwise");
    CapsuleParams P{c->nd.count, n, ks, kb, ka, node_mass, A0, P0};
    const int off = c->nd.count;
    const int id = (int)c->caps.size();
    std::vector<double2> zero(n, make_double2(0.0, 0.0));
    std::vector<int> zi(n, 0), cid(n, id);
    cudaStream_t s = c->stream;
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.X + off, xy, n * sizeof(double2), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.Xm1 + off, xy, n * sizeof(double2), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.uv + off, zero.data(), n * sizeof(double2), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.Fint + off, zero.data(), n * sizeof(double2), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.Fext + off, zero.data(), n * sizeof(double2), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.L0 + off, L0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.c0 + off, c0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.s0 + off, s0.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.age + off, zi.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.capid + off, cid.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->d_caps + id, &P, sizeof(P), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaStreamSynchronize(s));  // host staging vectors go out of scope
    c->caps.push_back(P);
    c->nd.count += n;
    if (n > c->max_n) c->max_n = n;
    // reference extent: the diagonal of the bounding box (an upper bound of the diameter,
    // so any rotation of the ring fits a square of this side)
    double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
    for (int a = 1; a < n; a++) {
        x0 = std::fmin(x0, xy[2 * a]); x1 = std::fmax(x1, xy[2 * a]);
        y0 = std::fmin(y0, xy[2 * a + 1]); y1 = std::fmax(y1, xy[2 * a + 1]);
    }
    const double ext = std::hypot(x1 - x0, y1 - y0);
    if (ext > c->max_extent) c->max_extent = ext;
    update_arcs(c);
    update_rep_grid(c);
    drop_graphs(c);  // launch shapes changed
    if (id_out) *id_out = id;
    return LBMIB_OK;
}

lbmib_status lbmib_field_ptr(lbmib_ctx* c, int field, void** ptr, int* pitch) {
    if (!c || !ptr || (field != LBMIB_FIELD_POPULATIONS && field != LBMIB_FIELD_FORCE))
        return c ? fail(c, LBMIB_ERR_ARG, "unknown field") : LBMIB_ERR_ARG;
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    *ptr = field == LBMIB_FIELD_POPULATIONS ? c->pops[c->cur] : (void*)c->fib[c->cur_fib];
    if (pitch) *pitch = field == LBMIB_FIELD_POPULATIONS ? c->L.pitch : c->L.nx;
    return LBMIB_OK;
}

lbmib_status lbmib_add_rigid(lbmib_ctx* c, const double* xy, int n, double mass, double inertia, int* id_out) {
    if (!c) return LBMIB_ERR_ARG;
    if (!xy || n < 3 || n > kMaxRing || !(mass > 0.0) || !(inertia > 0.0))
        return fail(c, LBMIB_ERR_ARG, "bad rigid particle arguments");
    // area centroid (shoelace, about the first vertex)
    double A2 = 0.0, sx = 0.0, sy = 0.0;
    for (int v = 0; v < n; v++) {
        const int r = v + 1 == n ? 0 : v + 1;
        const double ax = xy[2 * v] - xy[0], ay = xy[2 * v + 1] - xy[1];
        const double bx = xy[2 * r] - xy[0], by = xy[2 * r + 1] - xy[1];
        const double cr = ax * by - bx * ay;
        A2 += cr;
        sx += (ax + bx) * cr;
        sy += (ay + by) * cr;
    }
    if (!(A2 > 0.0)) return fail(c, LBMIB_ERR_ARG, "rigid particle ring must be counter-clockwise");
    const double cx = xy[0] + sx / (3.0 * A2), cy = xy[1] + sy / (3.0 * A2);
    int id = -1;
    lbmib_status st = lbmib_add_capsule(c, xy, n, 0.0, 0.0, 0.0, mass / n, &id);
    if (st != LBMIB_OK) return st;
    CapsuleParams& P = c->caps[id];
    P.rigid = 1;
    std::vector<double2> r0(n);
    for (int v = 0; v < n; v++) r0[v] = make_double2(xy[2 * v] - cx, xy[2 * v + 1] - cy);
    RigidBody B{};
    B.body[0] = B.prev[0] = cx;
    B.body[1] = B.prev[1] = cy;
    B.mass = mass;
    B.inertia = inertia;
    cudaStream_t s = c->stream;
    LBMIB_CUDA(c, cudaMemcpyAsync(c->d_caps + id, &P, sizeof(P), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.R0 + P.off, r0.data(), n * sizeof(double2), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.rb + id, &B, sizeof(B), cudaMemcpyHostToDevice, s));
    LBMIB_CUDA(c, cudaStreamSynchronize(s));
    c->nrigid++;
    if (id_out) *id_out = id;
    return LBMIB_OK;
}

lbmib_status lbmib_read_rigid(lbmib_ctx* c, int id, double* out) {
    if (!c || !out || id < 0 || id >= (int)c->caps.size() || !c->caps[id].rigid)
        return c ? fail(c, LBMIB_ERR_ARG, "not a rigid particle") : LBMIB_ERR_ARG;
    RigidBody B;
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    LBMIB_CUDA(c, cudaMemcpy(&B, c->nd.rb + id, sizeof(B), cudaMemcpyDeviceToHost));
    for (int j = 0; j < 6; j++) out[j] = B.body[j];
    for (int j = 0; j < 3; j++) out[6 + j] = B.load[j];
    return device_status(c);
}

lbmib_status lbmib_set_inflow(lbmib_ctx* c, const double* u_in, double rho_out) {
    if (!c) return LBMIB_ERR_ARG;
    Lat& L = c->L;
    if (!u_in) {
        L.inflow = 0;
        c->open = OpenBC{};
        drop_graphs(c);
        return LBMIB_OK;
    }
    if (L.nx < 5) return fail(c, LBMIB_ERR_ARG, "an open channel needs nx >= 5");
    if (!(rho_out > 0.5 && rho_out < 2.0)) return fail(c, LBMIB_ERR_ARG, "outlet density must be in (0.5, 2)");
    for (int y = 0; y < L.ny; y++)
        if (!(std::fabs(u_in[y]) < 0.3)) return fail(c, LBMIB_ERR_ARG, "inlet velocities must satisfy |u| < 0.3");
    LBMIB_CUDA(c, cudaMemcpyAsync(c->d_u_in, u_in, (size_t)L.ny * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    L.inflow = 1;
    c->open.u_in = c->d_u_in;
    c->open.drho_out = rho_out - 1.0;
    c->open.drho_outf = (float)c->open.drho_out;
    drop_graphs(c);
    return LBMIB_OK;
}

lbmib_status lbmib_set_repulsion(lbmib_ctx* c, double cutoff, double coeff) {
    if (!c || !(cutoff >= 0.0 && cutoff <= 16.0) || !(coeff >= 0.0))
        return fail(c, LBMIB_ERR_ARG, "repulsion: cut-off must be in [0, 16] and the coefficient >= 0");
    c->rep_rc = cutoff;
    c->rep_coeff = coeff > 0.0 ? coeff : 1e-4 / (8.0 * std::sqrt(2.0));   // Eq. 27 with dx = 1
    update_rep_grid(c);
    drop_graphs(c);
    return LBMIB_OK;
}

lbmib_status lbmib_set_capsule_positions(lbmib_ctx* c, int id, const double* xy) {
    if (!c || !xy || id < 0 || id >= (int)c->caps.size()) return LBMIB_ERR_ARG;
    if (c->caps[id].rigid) return fail(c, LBMIB_ERR_ARG, "a rigid particle moves only with its body state");
    const CapsuleParams& P = c->caps[id];
    std::vector<int> zi(P.n, 0);
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.X + P.off, xy, P.n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.Xm1 + P.off, xy, P.n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.age + P.off, zi.data(), P.n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBMIB_OK;
}

lbmib_status lbmib_step(lbmib_ctx* c, long long nsteps, lbmib_scheme scheme) {
    if (!c || nsteps < 0 || (scheme != LBMIB_KINEMATIC && scheme != LBMIB_DYNAMIC)) return LBMIB_ERR_ARG;
    if (scheme == LBMIB_KINEMATIC && c->nrigid > 0)
        return fail(c, LBMIB_ERR_STATE, "rigid particles move only with the Dynamic scheme");
    const int sc = scheme == LBMIB_DYNAMIC ? 1 : 0;
    if (c->timing || !c->use_graphs) {
        fork_ib(c, c->stream);
        enqueue_steps(c, scheme, nsteps, c->cur, c->cur_fib, c->stream, c->timing);
        join_ib(c, c->stream);
    } else {
        const int G = c->graph_steps > 0 ? c->graph_steps : 1;
        long long left = nsteps;
        while (left >= G) {
            cudaGraphExec_t& g = c->graphs[sc][c->cur][c->cur_fib];
            if (g && c->graph_len[sc][c->cur][c->cur_fib] != G) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
            if (!g) {
                lbmib_status st = capture(c, scheme, c->cur, c->cur_fib, G, &g, &c->graph_kernels[sc][c->cur][c->cur_fib]);
                if (st != LBMIB_OK) return st;
                c->graph_len[sc][c->cur][c->cur_fib] = G;
            }
            LBMIB_CUDA(c, cudaGraphLaunch(g, c->stream));
            c->launches += c->graph_kernels[sc][c->cur][c->cur_fib];
            // advance the host copy of the buffer parities by G steps
            for (int k = 0; k < G; k++) {
                if (!c->caps.empty()) c->cur_fib = 1 - c->cur_fib;
                c->cur = 1 - c->cur;
            }
            left -= G;
        }
        fork_ib(c, c->stream);
        enqueue_steps(c, scheme, left, c->cur, c->cur_fib, c->stream, false);
        join_ib(c, c->stream);
    }
    c->steps += nsteps;
    LBMIB_CUDA(c, cudaGetLastError());
    return LBMIB_OK;
}

lbmib_status lbmib_sync(lbmib_ctx* c) {
    if (!c) return LBMIB_ERR_ARG;
    return device_status(c);
}

lbmib_status lbmib_read_fields(lbmib_ctx* c, double* rho, double* ux, double* uy) {
    if (!c) return LBMIB_ERR_ARG;
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    by_storage(c->cfg.storage, [&](auto tag) {
        using S = decltype(tag);
        launch_macros<S>(c->pops[c->cur], c->L, c->open, c->fib[c->cur_fib], c->scratch, c->scratch + N,
                         c->scratch + 2 * N, c->stream);
    });
    c->launches++;
    LBMIB_CUDA(c, cudaGetLastError());
    double* h[3] = {rho, ux, uy};
    for (int k = 0; k < 3; k++)
        if (h[k])
            LBMIB_CUDA(c, cudaMemcpyAsync(h[k], c->scratch + k * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                                          c->stream));
    return device_status(c);
}

lbmib_status lbmib_read_populations(lbmib_ctx* c, double* f) {
    if (!c || !f) return LBMIB_ERR_ARG;
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    for (int i0 = 0; i0 < 9; i0 += 3) {
        by_storage(c->cfg.storage, [&](auto tag) {
            using S = decltype(tag);
            launch_populations<S>(c->pops[c->cur], c->L, c->open, i0, c->scratch, c->stream);
        });
        c->launches++;
        LBMIB_CUDA(c, cudaGetLastError());
        LBMIB_CUDA(c, cudaMemcpyAsync(f + i0 * N, c->scratch, 3 * N * sizeof(double), cudaMemcpyDeviceToHost,
                                      c->stream));
        LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return device_status(c);
}

lbmib_status lbmib_read_force_field(lbmib_ctx* c, double* fx, double* fy) {
    if (!c) return LBMIB_ERR_ARG;
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    if (fx) LBMIB_CUDA(c, cudaMemcpyAsync(fx, c->fib[c->cur_fib], N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (fy)
        LBMIB_CUDA(c, cudaMemcpyAsync(fy, c->fib[c->cur_fib] + N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return device_status(c);
}

lbmib_status lbmib_read_capsule(lbmib_ctx* c, int id, double* xy, double* vel, double* fint, double* fext) {
    if (!c || id < 0 || id >= (int)c->caps.size()) return LBMIB_ERR_ARG;
    const CapsuleParams& P = c->caps[id];
    const size_t b = P.n * sizeof(double2);
    if (xy) LBMIB_CUDA(c, cudaMemcpyAsync(xy, c->nd.X + P.off, b, cudaMemcpyDeviceToHost, c->stream));
    if (vel) LBMIB_CUDA(c, cudaMemcpyAsync(vel, c->nd.uv + P.off, b, cudaMemcpyDeviceToHost, c->stream));
    if (fint) LBMIB_CUDA(c, cudaMemcpyAsync(fint, c->nd.Fint + P.off, b, cudaMemcpyDeviceToHost, c->stream));
    if (fext) LBMIB_CUDA(c, cudaMemcpyAsync(fext, c->nd.Fext + P.off, b, cudaMemcpyDeviceToHost, c->stream));
    return device_status(c);
}

lbmib_status lbmib_observables(lbmib_ctx* c, int id, double out[8]) {
    if (!c || !out || id < 0 || id >= (int)c->caps.size()) return LBMIB_ERR_ARG;
    launch_observables(c->nd, (int)c->caps.size(), c->max_n, c->obs, c->stream);
    c->launches++;
    LBMIB_CUDA(c, cudaGetLastError());
    LBMIB_CUDA(c, cudaMemcpyAsync(out, c->obs + 8 * id, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return device_status(c);
}

lbmib_status lbmib_observables_all(lbmib_ctx* c, double* out) {
    if (!c || !out) return LBMIB_ERR_ARG;
    const int k = (int)c->caps.size();
    if (k == 0) return LBMIB_OK;
    launch_observables(c->nd, k, c->max_n, c->obs, c->stream);
    c->launches++;
    LBMIB_CUDA(c, cudaGetLastError());
    LBMIB_CUDA(c, cudaMemcpyAsync(out, c->obs, 8 * (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return device_status(c);
}

lbmib_status lbmib_interpolate(lbmib_ctx* c, const double* xy, int n, double* out) {
    if (!c || !xy || !out || n < 0 || n > c->cfg.max_nodes) return LBMIB_ERR_ARG;
    if (n == 0) return LBMIB_OK;
    LBMIB_CUDA(c, cudaMemcpyAsync(c->pts, xy, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    by_storage(c->cfg.storage, [&](auto tag) {
        using S = decltype(tag);
        launch_interp_points<S>(c->pops[c->cur], c->L, c->fib[c->cur_fib], c->pts, n, c->pts_out,
                                &c->ctr->status, c->stream);
    });
    c->launches++;
    LBMIB_CUDA(c, cudaGetLastError());
    LBMIB_CUDA(c, cudaMemcpyAsync(out, c->pts_out, 8 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return device_status(c);
}

lbmib_status lbmib_interpolate_noalloc(lbmib_ctx* c, const double* xy, int n, double* out) {
    if (!c || !xy || !out || n < 0) return LBMIB_ERR_ARG;
    if (n > kNoallocMaxPoints)
        return fail(c, LBMIB_ERR_ARG, "lbmib_interpolate_noalloc: n exceeds the static staging limit of 16384 points");
    if (n == 0) return LBMIB_OK;
    if (c->device < 0 || c->device >= kNoallocMaxDevices)
        return fail(c, LBMIB_ERR_ARG, "lbmib_interpolate_noalloc: device ordinal beyond the supported range");
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        base = g_noalloc_addr[c->device];
        if (!base) {
            // first call on this device: resolve the array's device address with the
            // context's device current (restored afterwards)
            int prev = 0;
            LBMIB_CUDA(c, cudaGetDevice(&prev));
            if (prev != c->device) LBMIB_CUDA(c, cudaSetDevice(c->device));
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_interp);
            if (prev != c->device) cudaSetDevice(prev);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(g_noalloc_interp)");
            g_noalloc_addr[c->device] = base = static_cast<double*>(p);
        }
    }
    double2* pts = reinterpret_cast<double2*>(base);
    double* res = base + 2 * kNoallocMaxPoints;
    LBMIB_CUDA(c, cudaMemcpyAsync(pts, xy, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    by_storage(c->cfg.storage, [&](auto tag) {
        using S = decltype(tag);
        launch_interp_points<S>(c->pops[c->cur], c->L, c->fib[c->cur_fib], pts, n, res, &c->ctr->status,
                                c->stream);
    });
    c->launches++;
    LBMIB_CUDA(c, cudaGetLastError());
    LBMIB_CUDA(c, cudaMemcpyAsync(out, res, 8 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return device_status(c);
}

// Snapshot: header | populations (latest post-collision) | last spread force | its
// touched-cell list | node arrays. Parities are normalised on load.
struct SnapHeader {
    char magic[8];
    int nx, ny, storage, ncaps, nnodes, count;
    long long steps;
};

size_t lbmib_state_bytes(const lbmib_ctx* c) {
    if (!c) return 0;
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)c->nd.count;
    return sizeof(SnapHeader) + 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage) + 2 * N * sizeof(double) +
           9 * (M > 0 ? M : 1) * sizeof(int) + M * (5 * sizeof(double2) + sizeof(int)) +
           c->caps.size() * sizeof(RigidBody);
}

lbmib_status lbmib_save_state(lbmib_ctx* c, void* buf, size_t bytes) {
    if (!c || !buf || bytes < lbmib_state_bytes(c)) return LBMIB_ERR_ARG;
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)c->nd.count;
    SnapHeader h{};
    memcpy(h.magic, "LBMIBv2", 8);
    h.nx = c->cfg.nx;
    h.ny = c->cfg.ny;
    h.storage = c->cfg.storage;
    h.ncaps = (int)c->caps.size();
    h.nnodes = (int)M;
    LBMIB_CUDA(c, cudaMemcpy(&h.count, &c->ctr->count[c->cur_fib], sizeof(int), cudaMemcpyDeviceToHost));
    h.steps = c->steps;
    char* p = (char*)buf;
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t pb = 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage);
    LBMIB_CUDA(c, cudaMemcpy(p, c->pops[c->cur], pb, cudaMemcpyDeviceToHost));
    p += pb;
    LBMIB_CUDA(c, cudaMemcpy(p, c->fib[c->cur_fib], 2 * N * sizeof(double), cudaMemcpyDeviceToHost));
    p += 2 * N * sizeof(double);
    const size_t lb = 9 * (M > 0 ? M : 1) * sizeof(int);
    LBMIB_CUDA(c, cudaMemcpy(p, c->list[c->cur_fib], lb, cudaMemcpyDeviceToHost));
    p += lb;
    double2* arrs[5] = {c->nd.X, c->nd.Xm1, c->nd.uv, c->nd.Fint, c->nd.Fext};
    for (auto* a : arrs) {
        LBMIB_CUDA(c, cudaMemcpy(p, a, M * sizeof(double2), cudaMemcpyDeviceToHost));
        p += M * sizeof(double2);
    }
    LBMIB_CUDA(c, cudaMemcpy(p, c->nd.age, M * sizeof(int), cudaMemcpyDeviceToHost));
    p += M * sizeof(int);
    LBMIB_CUDA(c, cudaMemcpy(p, c->nd.rb, c->caps.size() * sizeof(RigidBody), cudaMemcpyDeviceToHost));
    return device_status(c);
}

lbmib_status lbmib_load_state(lbmib_ctx* c, const void* buf, size_t bytes) {
    if (!c || !buf || bytes < sizeof(SnapHeader)) return LBMIB_ERR_ARG;
    SnapHeader h;
    memcpy(&h, buf, sizeof(h));
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)c->nd.count;
    if (memcmp(h.magic, "LBMIBv2", 8) != 0 || h.nx != c->cfg.nx || h.ny != c->cfg.ny ||
        h.storage != (int)c->cfg.storage || h.ncaps != (int)c->caps.size() || h.nnodes != (int)M ||
        bytes < lbmib_state_bytes(c))
        return fail(c, LBMIB_ERR_STATE, "snapshot does not match this context");
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    const char* p = (const char*)buf + sizeof(h);
    c->cur = 0;
    c->cur_fib = 0;
    const size_t pb = 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage);
    LBMIB_CUDA(c, cudaMemcpy(c->pops[0], p, pb, cudaMemcpyHostToDevice));
    p += pb;
    LBMIB_CUDA(c, cudaMemset(c->fib[1], 0, 2 * N * sizeof(double)));
    LBMIB_CUDA(c, cudaMemcpy(c->fib[0], p, 2 * N * sizeof(double), cudaMemcpyHostToDevice));
    p += 2 * N * sizeof(double);
    const size_t lb = 9 * (M > 0 ? M : 1) * sizeof(int);
    LBMIB_CUDA(c, cudaMemcpy(c->list[0], p, lb, cudaMemcpyHostToDevice));
    p += lb;
    double2* arrs[5] = {c->nd.X, c->nd.Xm1, c->nd.uv, c->nd.Fint, c->nd.Fext};
    for (auto* a : arrs) {
        LBMIB_CUDA(c, cudaMemcpy(a, p, M * sizeof(double2), cudaMemcpyHostToDevice));
        p += M * sizeof(double2);
    }
    LBMIB_CUDA(c, cudaMemcpy(c->nd.age, p, M * sizeof(int), cudaMemcpyHostToDevice));
    p += M * sizeof(int);
    LBMIB_CUDA(c, cudaMemcpy(c->nd.rb, p, c->caps.size() * sizeof(RigidBody), cudaMemcpyHostToDevice));
    // fresh claims: no node carries a stamp that a coming patch will use
    LBMIB_CUDA(c, cudaMemset(c->mark, 0, N * sizeof(int)));
    DevCounters ctr{};
    ctr.count[0] = h.count;
    LBMIB_CUDA(c, cudaMemcpy(c->ctr, &ctr, sizeof(ctr), cudaMemcpyHostToDevice));
    c->steps = h.steps;
    drop_graphs(c);
    return LBMIB_OK;
}

lbmib_status lbmib_set_option(lbmib_ctx* c, int option, long long value) {
    if (!c) return LBMIB_ERR_ARG;
    switch (option) {
        case LBMIB_OPT_GRAPHS: c->use_graphs = value != 0; break;
        case LBMIB_OPT_TIMING: c->timing = value != 0; break;
        case LBMIB_OPT_OVERLAP:
            if (value < -1 || value > 1) return fail(c, LBMIB_ERR_ARG, "overlap must be -1, 0 or 1");
            c->overlap = (int)value;
            drop_graphs(c);
            break;
        case LBMIB_OPT_GRAPH_STEPS:
            if (value < 1 || value > 4096) return fail(c, LBMIB_ERR_ARG, "graph steps out of range");
            c->graph_steps = (int)value;
            drop_graphs(c);
            break;
        case LBMIB_OPT_FP16_SCALE:
            if (value < 0 || value > 14) return fail(c, LBMIB_ERR_ARG, "FP16 scale exponent out of range");
            if (c->cfg.storage == LBMIB_FP16) {
                c->L.scale = (float)std::ldexp(1.0, (int)value);
                c->L.inv_scale = 1.0f / c->L.scale;
                drop_graphs(c);
            }
            break;
        case LBMIB_OPT_LATTICE_VARIANT:
            c->lattice_variant = (int)value;
            drop_graphs(c);
            break;
        case LBMIB_OPT_IB_FP64:
            if (value < 0 || value > 1) return fail(c, LBMIB_ERR_ARG, "IB FP64 must be 0 or 1");
            c->ib_fp64 = value != 0 && c->cfg.storage != LBMIB_FP64;
            drop_graphs(c);
            break;
        case LBMIB_OPT_FUSE_IB:
            if (value < 0 || value > 1) return fail(c, LBMIB_ERR_ARG, "fuse must be 0 or 1");
            c->fuse_ib = value != 0;
            drop_graphs(c);
            break;
        case LBMIB_OPT_ARCS:
            if (value < 0 || value > kMaxArcs) return fail(c, LBMIB_ERR_ARG, "arcs must be in [0, 8]");
            c->arcs_opt = (int)value;
            update_arcs(c);
            drop_graphs(c);
            break;
        default: return fail(c, LBMIB_ERR_ARG, "unknown option");
    }
    return LBMIB_OK;
}

// Fold the recorded events into the totals (the lattice pairs, then the IB events that
// refer to them) and recycle them.
static lbmib_status fold_timing(lbmib_ctx* c) {
    LBMIB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (const auto& e : c->ev_ib) {
        float mp = 0.0f, mi = 0.0f;
        LBMIB_CUDA(c, cudaEventElapsedTime(&mp, c->ev_pool[e.lat].second, e.patch_end));
        LBMIB_CUDA(c, cudaEventElapsedTime(&mi, e.patch_end, e.ib_end));
        c->timed_patch_ms += mp;
        c->timed_ib_ms += mi;
        c->timed_ib_steps++;
        c->ev_ib_free.push_back({e.patch_end, e.ib_end});
    }
    c->ev_ib.clear();
    for (size_t k = 0; k < c->ev_used; k++) {
        float ms = 0.0f;
        LBMIB_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[k].first, c->ev_pool[k].second));
        c->timed_ms += ms;
        c->timed_launches++;
    }
    c->ev_used = 0;
    return LBMIB_OK;
}

lbmib_status lbmib_ib_kernel_time(lbmib_ctx* c, double* patch_ms, double* ib_ms, long long* steps,
                                  long long* listed, int reset) {
    if (!c) return LBMIB_ERR_ARG;
    const lbmib_status st = fold_timing(c);
    if (st != LBMIB_OK) return st;
    if (patch_ms) *patch_ms = c->timed_patch_ms;
    if (ib_ms) *ib_ms = c->timed_ib_ms;
    if (steps) *steps = c->timed_ib_steps;
    if (listed) {
        int n = 0;
        LBMIB_CUDA(c, cudaMemcpy(&n, &c->ctr->count[c->cur_fib], sizeof(int), cudaMemcpyDeviceToHost));
        *listed = n;
    }
    if (reset) {
        c->timed_patch_ms = c->timed_ib_ms = 0.0;
        c->timed_ib_steps = 0;
    }
    return LBMIB_OK;
}

lbmib_status lbmib_kernel_time(lbmib_ctx* c, double* total_ms, long long* launches, int reset) {
    if (!c) return LBMIB_ERR_ARG;
    const lbmib_status st = fold_timing(c);
    if (st != LBMIB_OK) return st;
    if (total_ms) *total_ms = c->timed_ms;
    if (launches) *launches = c->timed_launches;
    if (reset) {
        c->timed_ms = 0.0;
        c->timed_launches = 0;
    }
    return LBMIB_OK;
}

long long lbmib_launch_count(const lbmib_ctx* c) { return c ? c->launches : 0; }

double lbmib_bytes_per_update(const lbmib_ctx* c) {
    return c ? 18.0 * (double)storage_bytes(c->cfg.storage) : 0.0;
}

}  // extern "C"
