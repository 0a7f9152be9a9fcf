// Immersed-boundary kernels: MLS interpolation and spreading (Eq. 8-9, Section 2.3
// step 3, Section 2.4 step iii), membrane forces (Eq. 10-14), hydrodynamic tractions
// (Eq. 15-16), and the node updates of the Dynamic (Eq. 21-24) and Kinematic (Eq. 25)
// schemes. Coclite et al., arXiv:1903.03356.
//
// Every kernel here runs `arcs` CTAs per capsule, each owning one arc of the ring (the
// whole ring when arcs = 1; more arcs when the capsules are too few to fill the GPU).
// The CTA stages its arc in shared memory, takes the bounding box of the arc (plus the
// reach of the supports, and of the probes when it needs them) and fills a shared tile
// with the lattice moments of every node in the box once (nine pulls per node). Node and probe interpolations then read
// that tile instead of re-gathering 81 populations each, and the spread accumulates
// into a shared force tile that is flushed once per touched node (one global atomic
// per node instead of one per marker and support point). A capsule whose box does not
// fit the tile budget takes the same path with global pulls and global atomics. The
// kernels that need the enclosed area run each capsule's CTAs as a thread-block cluster
// and add the arcs' partial sums through distributed shared memory.
// Positions, velocities, forces and reference lengths are double in every storage mode;
// in FP32/FP16 modes the MLS weights, their solve and the weighted sums are float. The
// two Dynamic IB kernels are bound to 6 CTAs per SM: their FP64 work issues at 2 per SM
// per cycle on GB300, and more resident CTAs keep that pipe fed.
#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <utility>

#include "ring.cuh"

namespace cg = cooperative_groups;

namespace lbmib {

size_t capsule_smem_bytes(int max_n) { return ring_smem_bytes(max_n); }

// Reduction scratch of the 128-thread capsule kernels (4 warps x 8 doubles): smaller
// scratch lets seven CTAs share a multiprocessor's shared memory.
constexpr int kRedIB = 4 * 8;

// Fill the moment tile from the populations (nine pulls per node, row by row), two
// nodes per thread and pass with both nodes' pulls issued before either is reduced: the
// fill waits on memory latency, and this halves its round trips.
template <typename S>
__device__ void fill_moments(Tile<typename St<S>::C>& t, const S* __restrict__ src, const Lat& L,
                             const double* __restrict__ fib) {
    using C = typename St<S>::C;
    const int cells = t.w * t.h;
    for (int k = threadIdx.x; k < cells; k += 2 * blockDim.x) {
        const int k1 = k + blockDim.x;
        const int j0 = k / t.w, i0 = k - j0 * t.w;
        const int k1c = k1 < cells ? k1 : k;   // a missing second node repeats the first
        const int j1 = k1c / t.w, i1 = k1c - j1 * t.w;
        const Mom<C> m0 = node_moments<S>(src, L, fib, wrapi(t.x0 + i0, L.nx), support_row(L, t.y0 + j0));
        const Mom<C> m1 = node_moments<S>(src, L, fib, wrapi(t.x0 + i1, L.nx), support_row(L, t.y0 + j1));
        t.drho[k] = m0.drho;
        t.ux[k] = m0.ux;
        t.uy[k] = m0.uy;
        if (k1 < cells) {
            t.drho[k1] = m1.drho;
            t.ux[k1] = m1.ux;
            t.uy[k1] = m1.uy;
        }
    }
}

__device__ __forceinline__ void touch(const Spread& sp, int cell) {
    const int p = atomicAdd(sp.count, 1);
    if (p < sp.capacity) sp.list[p] = cell;
    else atomicOr(sp.status, kStatList);
}

// Add the force tile to the lattice force field and record the touched nodes. The
// tile's nonzero nodes are collected in shared memory first and appended with one global
// reservation per capsule, so that the list counter is not a hot spot, and nothing in
// the loop waits on a global round trip (the force adds are fire-and-forget). A node
// that the tiles of several capsules cover is listed once by each: the patch forces it
// once (its first entry claims it) and clears its force once per entry, and the list
// still holds at most 9 entries per vertex.
// Collective (all threads); the moment arrays are dead by now and hold the scratch.
template <typename C>
__device__ void flush_forces(const Tile<C>& t, const Lat& L, const Spread& sp, int* s_count) {
    const long long N = (long long)L.nx * L.ny;
    const int cells = t.w * t.h;
    if (threadIdx.x == 0) *s_count = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        const C cx = t.fx[k], cy = t.fy[k];   // zero test before the widening (exact either way)
        if (cx == C(0) && cy == C(0)) continue;
        const int j = k / t.w, i = k - j * t.w;
        const int cell = support_row(L, t.y0 + j) * L.nx + wrapi(t.x0 + i, L.nx);
        atomicAdd(sp.fib + cell, (double)cx);
        atomicAdd(sp.fib + N + cell, (double)cy);
        t.cells[atomicAdd(s_count, 1)] = cell;
    }
    __syncthreads();
    const int nnew = *s_count;
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = nnew > 0 ? atomicAdd(sp.count, nnew) : 0;
    __syncthreads();
    for (int k = threadIdx.x; k < nnew; k += blockDim.x) {
        const int p = s_base + k;
        if (p < sp.capacity) sp.list[p] = t.cells[k];
        else atomicOr(sp.status, kStatList);
    }
}

// Interpolation (Eq. 8) with the shape functions m from the tile, or from the
// populations when the capsule has no tile.
template <typename S, bool GRAD>
__device__ __forceinline__ bool interp_with(const MlsW<typename St<S>::C>& m, const Tile<typename St<S>::C>& t,
                                            const S* __restrict__ src, const Lat& L, const double* __restrict__ fib,
                                            InterpT<typename St<S>::C>& o) {
    using C = typename St<S>::C;
    if (!t.use) return mls_interp_with<S, GRAD>(m, src, L, fib, o);
    if (!t.holds(m.cx, m.cy)) {
        // only a runaway point (already moved to the origin) can leave the box: flag it
        mls_interp_with<S, GRAD>(m, src, L, fib, o);
        return false;
    }
    mls_apply<C, GRAD>(m, [&](int a, int b) {
        const int k = t.index(m.cx + a - 1, m.cy + b - 1);
        Mom<C> q;
        q.drho = t.drho[k];
        q.ux = t.ux[k];
        q.uy = t.uy[k];
        return q;
    }, o);
    return m.ok;
}

// Interpolation (Eq. 8) at (X, Y) from the tile, or from the populations when the
// capsule has no tile.
template <typename S, bool GRAD>
__device__ __forceinline__ bool interp_at(const Tile<typename St<S>::C>& t, const S* __restrict__ src, const Lat& L,
                                          const double* __restrict__ fib, double X, double Y,
                                          InterpT<typename St<S>::C>& o) {
    return interp_with<S, GRAD>(mls_setup<typename St<S>::C>(L, X, Y), t, src, L, fib, o);
}

// Spread c * F with the shape functions m (step 3 / step iii): into the force tile, or
// straight into the lattice field when the capsule has no tile.
template <typename C>
__device__ __forceinline__ bool spread_with(const MlsW<C>& m, Tile<C>& t, const Lat& L, const Spread& sp,
                                            C Fx, C Fy, C c) {
    const long long N = (long long)L.nx * L.ny;
    const bool in_tile = t.holds(m.cx, m.cy);
    const C cFx = c * Fx, cFy = c * Fy;
#pragma unroll
    for (int b = 0; b < 3; b++) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const C phi = m.phi(a, b);
            if (in_tile) {
                const int k = t.index(m.cx + a - 1, m.cy + b - 1);
                atomicAdd(t.fx + k, phi * cFx);
                atomicAdd(t.fy + k, phi * cFy);
            } else {
                const double w = (double)c * (double)phi;
                const int cell = support_row(L, m.cy + b - 1) * L.nx + wrapi(m.cx + a - 1, L.nx);
                atomicAdd(sp.fib + cell, w * (double)Fx);
                atomicAdd(sp.fib + N + cell, w * (double)Fy);
                touch(sp, cell);
            }
        }
    }
    return m.ok && (in_tile || !t.use);
}

// ---------------------------------------------------------------------------------
// Arcs. A launch gives each capsule `arcs` CTAs (a thread-block cluster when the kernel
// needs the enclosed area): CTA `rank` owns the vertices [v0, v0 + m) of an even split
// of the ring and stages them in slots kHalo .. kHalo + m - 1, with kHalo neighbours on
// each side (wrapping around the ring). Its tile covers only its arc. With arcs = 1 the
// one arc is the whole ring.
// ---------------------------------------------------------------------------------
struct Arc {
    int cap, rank;  // capsule, position among its CTAs
    int n, v0, m;   // ring size, first own vertex, own vertices
    double2 X0;     // X_0, the origin of the area sums
    // node index (within the capsule) of staged slot li
    __device__ __forceinline__ int node(int li) const { return (v0 - kHalo + li + n) % n; }
};

// Load this CTA's capsule and stage its arc (with the halo slots when `halo`); false
// (after flagging) when the capsule's parameters are out of range, which every CTA of
// the capsule sees alike.
__device__ __forceinline__ bool load_arc(const Nodes& nd, const CapSmem& sm, int max_n, int arcs, bool halo,
                                         CapsuleParams& P, Arc& a, unsigned* status) {
    const int cap = blockIdx.x / arcs, rank = blockIdx.x - cap * arcs;
    P = nd.caps[cap];
    if (P.n < 3 || P.n > max_n || P.off < 0 || P.off + P.n > nd.count) {
        if (threadIdx.x == 0) atomicOr(status, kStatRing);
        return false;
    }
    const int chunk = (P.n + arcs - 1) / arcs;
    a.cap = cap;
    a.rank = rank;
    a.n = P.n;
    a.v0 = rank * chunk;
    a.m = max(0, min(P.n - a.v0, chunk));
    a.X0 = nd.X[P.off];
    const int lo = halo ? 0 : kHalo, hi = a.m == 0 ? lo : a.m + kHalo + (halo ? kHalo : 0);
    for (int li = lo + threadIdx.x; li < hi; li += blockDim.x) sm.X[li] = nd.X[P.off + a.node(li)];
    __syncthreads();
    return true;
}

// Sum of a CTA-uniform value over the CTAs of this capsule's cluster, added in rank
// order so that every CTA gets the same bits. Collective over the cluster.
template <int K>
__device__ __forceinline__ void cluster_total(double (&v)[K], int arcs) {
    if (arcs == 1) return;
    __shared__ double part[K];
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < K; j++) part[j] = v[j];
    cl.sync();
#pragma unroll
    for (int j = 0; j < K; j++) {
        double t = 0.0;
        for (int r = 0; r < arcs; r++) t += cl.map_shared_rank(part, r)[j];
        v[j] = t;
    }
    cl.sync();   // no CTA leaves while another still reads its partials
}
__device__ __forceinline__ double cluster_total(double v, int arcs) {
    double t[1] = {v};
    cluster_total<1>(t, arcs);
    return t[0];
}

// Velocity of the rigid-body motion of body state b at point X.
__device__ __forceinline__ double2 rigid_velocity(const double* b, double2 X) {
    return make_double2(b[3] - b[5] * (X.y - b[1]), b[4] + b[5] * (X.x - b[0]));
}

// A whole ring's halo slots repeat its own last and first vertex: copy their terms
// (and the element tractions when `ext`), double or single-precision (F32) ones.
// Collective; ends with a barrier.
template <bool F32 = false>
__device__ __forceinline__ void copy_halo_terms(const CapSmem& sm, int m, bool ext) {
    if (F32 && threadIdx.x == 0) {
        const int lo = kHalo - 1, last = kHalo + m - 1, hi = kHalo + m, first = kHalo;
        RingF* R = ring_f(sm);
        R[lo] = R[last];
        R[hi] = R[first];
        if (ext) ext_f(sm)[lo] = ext_f(sm)[last];
    } else if (threadIdx.x == 0) {
        const int lo = kHalo - 1, last = kHalo + m - 1, hi = kHalo + m, first = kHalo;
        sm.sst[lo] = sm.sst[last];
        sm.bs[lo] = sm.bs[last];
        sm.bdl[lo] = sm.bdl[last];
        sm.bdr[lo] = sm.bdr[last];
        if (ext) sm.ext[lo] = sm.ext[last];
        sm.sst[hi] = sm.sst[first];
        sm.bs[hi] = sm.bs[first];
        sm.bdl[hi] = sm.bdl[first];
        sm.bdr[hi] = sm.bdr[first];
    }
    __syncthreads();
}

// Resident CTAs per SM the Dynamic IB kernels are compiled for: 6 in single precision
// (80 registers; their FP64 work issues at 2 per SM per cycle on GB300 and more CTAs keep
// that pipe fed), the register file's own limit in double, which would spill at 6.
template <typename S>
constexpr int dyn_min_blocks() {
    return sizeof(typename St<S>::C) == 4 ? 8 : 1;
}

// An odd step coprime to m, about a quarter of m (1 for short arcs): j -> j * hop mod m
// visits every vertex once and puts consecutive j far apart on the ring.
__device__ __forceinline__ int ring_hop(int m) {
    if (m < 64) return 1;
    for (int h = (m / 4) | 1; h < m / 2; h += 2) {
        int a = h, b = m;
        while (b) {
            const int r = a % b;
            a = b;
            b = r;
        }
        if (a == 1) return h;
    }
    return 1;
}

// ---------------------------------------------------------------------------------
// Dynamic IB (Section 2.3.2), steps 1-3: U = I(u^n) of the populations before any IB
// force (rho u = sum f e + g/2; the step's IB force is the unknown of the direct forcing),
// F_l = u_v - U, spread with c_l = (l_left + l_right)/2. U is kept per vertex: it is also
// the tentative velocity of the step's Eq. 23 (the fluid velocity at time t). First step
// of a vertex: u_v = U and X^{-1} = X^0 - U.
// ---------------------------------------------------------------------------------
// Steps 1-3 on a staged arc whose tile holds the moments of the lattice state and zeroed
// force accumulators (collective; starts with a barrier-ordered pass over the element
// lengths). Returns false when a support left the channel or the tile. FRAMED (single
// precision): the support frames at X^n are already stored (by the previous update).
template <typename S, bool RIGID, bool FRAMED = false>
__device__ __forceinline__ bool dyn_spread(const S* __restrict__ src, const Lat& L, const Nodes& nd, const CapsuleParams& P, const Arc& a, const CapSmem& sm,
                                           Tile<typename St<S>::C>& t, const Spread& sp) {
    using C = typename St<S>::C;
    constexpr bool F32 = sizeof(C) == 4;   // single precision: lengths and forces in float
    // lengths of the elements on both sides of every own vertex (c_l of reading R4). FRAMED
    // (single precision, right after this CTA's node update): the staged slots still hold
    // X^n, with the float edge vectors of X^n and the float increments X^{n+1} - X^n, so
    // the edges of X^{n+1} are e + (d_{v+1} - d_v) in float, to the float rounding of the
    // double differences they replace.
    for (int e = threadIdx.x; e < (a.m > 0 ? a.m + 1 : 0); e += blockDim.x) {
        const int li = kHalo - 1 + e;
        if constexpr (FRAMED && F32) {
            const float2 ev = ring_f(sm)[li].e, d0 = xd_f(sm)[li], d1 = xd_f(sm)[li + 1];
            const float dx = ev.x + (d1.x - d0.x), dy = ev.y + (d1.y - d0.y);
            len_f(sm)[li] = sqrtf(dx * dx + dy * dy);
        } else {
            const double2 d = sm.X[li + 1] - sm.X[li];
            if constexpr (F32) {
                const float dx = (float)d.x, dy = (float)d.y;
                len_f(sm)[li] = sqrtf(dx * dx + dy * dy);
            } else {
                sm.sst[li] = sqrt(d.x * d.x + d.y * d.y);
            }
        }
    }
    __syncthreads();
    bool ok = true;
    // the lanes of a warp take vertices `hop` apart on the ring (a bijection of 0..m-1):
    // their 3x3 supports then rarely share a tile cell, and the shared-memory atomics of
    // the spread rarely collide within an instruction
    const int hop = ring_hop(a.m);
    for (int j = threadIdx.x; j < a.m; j += blockDim.x) {
        const int k = (int)((long long)j * hop % a.m);
        const int li = kHalo + k, g = P.off + a.v0 + k;
        // shape functions at X^n: used for U, for the spread, and by this step's update
        MlsW<C> w;
        if constexpr (FRAMED && sizeof(C) == 4) {   // the frame the update of this CTA left
            const int2 fc = frame_c_f(sm)[li];
            const float2 fd = frame_d_f(sm)[li];
            w = mls_from_frame<C>(L, MlsFrame{fc.x, fc.y, fd.x, fd.y});
        } else {
            const double2 Xv = sm.X[li];
            w = mls_setup<C>(L, Xv.x, Xv.y);
            store_mls<C>(nd.mls, g, w);
        }
        InterpT<C> o;
        ok &= interp_with<S, false>(w, t, src, L, nullptr, o);
        // U as computed: float for single precision, double otherwise
        if constexpr (F32) u_f(nd)[g] = make_float2(o.ux, o.uy);
        else nd.U[g] = make_double2((double)o.ux, (double)o.uy);
        double2 uv;
        if (RIGID && P.rigid) {
            uv = rigid_velocity(nd.rb[a.cap].body, sm.X[li]);   // the body's motion (Section 2.3.1)
        } else if (FRAMED && F32) {
            const float2 u = uv_next_f(sm)[li];   // the update of this CTA left it (float is all F needs)
            uv = make_double2(u.x, u.y);
        } else {
            uv = nd.uv[g];
            if (!FRAMED && nd.age[g] == 0) {   // a vertex's first step (never a fused one)
                uv = make_double2((double)o.ux, (double)o.uy);
                nd.uv[g] = uv;
                nd.Xm1[g] = sm.X[li] - uv;
            }
        }
        const double Ux = (double)o.ux, Uy = (double)o.uy;
        if constexpr (F32) {
            const float cl = 0.5f * (len_f(sm)[li - 1] + len_f(sm)[li]);
            const float Fx = (float)uv.x - o.ux, Fy = (float)uv.y - o.uy;
            if (nd.Flc) nd.Flc[g] = make_double2((double)(cl * Fx), (double)(cl * Fy));
            ok &= spread_with<C>(w, t, L, sp, Fx, Fy, cl);
        } else {
            const double cl = 0.5 * (sm.sst[li - 1] + sm.sst[li]);
            if (nd.Flc) nd.Flc[g] = make_double2(cl * (uv.x - Ux), cl * (uv.y - Uy));
            ok &= spread_with<C>(w, t, L, sp, uv.x - Ux, uv.y - Uy, cl);
        }
    }
    return ok;
}

template <typename S, bool RIGID>
__global__ void __launch_bounds__(128, dyn_min_blocks<S>()) k_dyn_force_spread(const S* __restrict__ src, Lat L,
                                                          Nodes nd, int max_n,
                                                          int arcs, int tile_cells, Spread sp, unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, arc_slots(max_n, arcs), kRedIB);
    CapsuleParams P;
    Arc a;
    if (!load_arc(nd, sm, max_n, arcs, true, P, a, status)) return;
    Tile<C> t = make_tile<C>(sm, kHalo, kHalo + a.m, 1, tile_cells, true, true);
    if (t.use) {
        fill_moments<S>(t, src, L, nullptr);
        zero_forces<C>(t);
    }
    const bool ok = dyn_spread<S, RIGID>(src, L, nd, P, a, sm, t, sp);
    __syncthreads();
    if (t.use) flush_forces<C>(t, L, sp, reinterpret_cast<int*>(sm.red));
    if (!ok) atomicOr(status, kStatSupport);
}

// Rigid particle, after its load is summed (Section 2.3.1): accelerations F/m and M/I,
// Eq. 19-20 for the velocities, the same backward form for the centre and the angle,
// and the markers X_v = c + R(theta) r_v moving with u + omega x (X_v - c). Every CTA of
// the particle computes the same update from the same totals; the first stores it.
__device__ void rigid_update(const Nodes& nd, const CapsuleParams& P, const Arc& a, const CapSmem& sm,
                             const double* body, const double* prev, const double (&sums)[3]) {
    const RigidBody& B = nd.rb[a.cap];
    const double acc[3] = {sums[0] / B.mass, sums[1] / B.mass, sums[2] / B.inertia};
    double next[6];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        next[3 + j] = (2.0 / 3.0) * (2.0 * body[3 + j] - 0.5 * prev[3 + j] + acc[j]);
        next[j] = (2.0 / 3.0) * (2.0 * body[j] - 0.5 * prev[j] + next[3 + j]);
    }
    double sn, cs;
    sincos(next[2], &sn, &cs);
    for (int k = threadIdx.x; k < a.m; k += blockDim.x) {
        const int li = kHalo + k, g = P.off + a.v0 + k;
        const double2 r0 = nd.R0[g];
        const double rx = cs * r0.x - sn * r0.y, ry = sn * r0.x + cs * r0.y;
        nd.Xm1[g] = sm.X[li];
        nd.X[g] = make_double2(next[0] + rx, next[1] + ry);
        nd.uv[g] = make_double2(next[3] - next[5] * ry, next[4] + next[5] * rx);
        nd.Fint[g] = make_double2(0.0, 0.0);
        nd.Fext[g] = 0.5 * (sm.ext[li] + sm.ext[li - 1]);
        nd.age[g] += 1;
    }
    if (a.rank == 0 && threadIdx.x == 0) {
        RigidBody& W = nd.rb[a.cap];
#pragma unroll
        for (int j = 0; j < 6; j++) {
            W.prev[j] = body[j];
            W.body[j] = next[j];
        }
        for (int j = 0; j < 3; j++) W.load[j] = sums[j];
    }
}

// Dynamic IB steps 7-8: probe tractions (Eq. 15-16) on the updated populations (before
// any IB force, as in step 1), internal forces (Eq. 11, 13, 14), Verlet position (Eq. 23)
// with the tentative velocity U of step 1, and BDF2 velocity (Eq. 24).
// With arcs > 1 the capsule's CTAs form a cluster: the enclosed area is summed over it,
// and its barrier also orders every CTA's reads of X^n (own and halo) before any CTA
// writes X^{n+1}.
// Steps 5-8 on a staged arc (m own vertices; 0 for a rigid particle's CTAs) whose tile
// holds the moments of the lattice state after the fluid update. Collective over the
// capsule's cluster when arcs > 1. Returns false when a support left the channel or the
// tile. NEXT (single precision, one CTA per ring): also store each vertex's support frame
// at X^{n+1}, found from its frame at X^n and the increment, for the next step's spread.
template <typename S, bool NEXT = false>
__device__ __forceinline__ bool dyn_update(const S* __restrict__ dst, const Lat& L, const Nodes& nd, const CapsuleParams& P, const Arc& a, const CapSmem& sm,
                                           const Tile<typename St<S>::C>& t, int arcs, int m) {
    using C = typename St<S>::C;
    bool ok = true;
    double area2[1] = {0.0};
    float area2f[1] = {0.0f};   // single precision
    const C nu = C(L.nu);
    // task k < m: own vertex kHalo+k (velocity, ring terms, area) and its element
    // (tractions). A split ring adds two tasks for the halo: element and ring terms of
    // slot kHalo-1, ring terms of slot kHalo+m. A whole ring copies them instead.
    const bool split = m > 0 && m < a.n;   // an arc without vertices has no tasks
    constexpr bool F32 = sizeof(C) == 4;   // single precision: membrane terms and tractions in float
    for (int k = threadIdx.x; k < (split ? m + 2 : m); k += blockDim.x) {
        const int li = k < m ? kHalo + k : (k == m ? kHalo - 1 : kHalo + m);
        if constexpr (F32) {
            vertex_terms_f(sm, P, nd, li - 1, li, li + 1, P.off + a.node(li));
            if (k == m + 1) continue;
            // the vertex's shape functions at X^n (stored by this step's spread kernel) place
            // the probes of its element in float
            const MlsW<C> w = load_mls<C>(L, nd.mls, P.off + a.node(li));
            if (k < m && P.ka != 0.0) {
                // the area term (X_v - X_0) x (X_{v+1} - X_0) = (X_v - X_0) x e_v, in float:
                // its rounding is of the order of the float membrane terms'
                const double2 Xv = sm.X[li];
                const float2 e = ring_f(sm)[li].e;
                area2f[0] += (float)(Xv.x - a.X0.x) * e.y - (float)(Xv.y - a.X0.y) * e.x;
            }
            // element li: probes at the centroid +/- 1.2 n+ (Section 2.2.2)
            const float2 e = ring_f(sm)[li].e;
            const float e2 = e.x * e.x + e.y * e.y, rl = rsqrtf(e2);
            const float nx = e.y * rl, ny = -e.x * rl;
            InterpT<C> op, om;
            ok &= interp_with<S, true>(mls_near<C>(L, w, 0.5f * e.x + 1.2f * nx, 0.5f * e.y + 1.2f * ny), t, dst,
                                       L, nullptr, op);
            ok &= interp_with<S, true>(mls_near<C>(L, w, 0.5f * e.x - 1.2f * nx, 0.5f * e.y - 1.2f * ny), t, dst,
                                       L, nullptr, om);
            const C mp = op.rho * nu, mm = om.rho * nu;
            const C txx = C(2) * (mp * op.dudx - mm * om.dudx);
            const C tyy = C(2) * (mp * op.dvdy - mm * om.dvdy);
            const C txy = mp * (op.dudy + op.dvdx) - mm * (om.dudy + om.dvdx);
            const C dp = op.p - om.p;
            const float len = e2 * rl;
            ext_f(sm)[li] = make_float2((-dp * nx + txx * nx + txy * ny) * len, (-dp * ny + txy * nx + tyy * ny) * len);
            continue;
        }
        vertex_terms(sm, P, nd, li - 1, li, li + 1, P.off + a.node(li));
        if (k == m + 1) continue;
        const double2 Xv = sm.X[li], Xr = sm.X[li + 1];
        if (k < m) area2[0] += area_term(a.X0, Xv, Xr);
        // element li: probes at the centroid +/- 1.2 n+ (Section 2.2.2)
        const double2 d = Xr - Xv;
        const double rl = rsqrt(d.x * d.x + d.y * d.y);
        const double npx = d.y * rl, npy = -d.x * rl;
        const double cx = 0.5 * (Xv.x + Xr.x), cy = 0.5 * (Xv.y + Xr.y);
        InterpT<C> op, om;
        ok &= interp_at<S, true>(t, dst, L, nullptr, cx + 1.2 * npx, cy + 1.2 * npy, op);
        ok &= interp_at<S, true>(t, dst, L, nullptr, cx - 1.2 * npx, cy - 1.2 * npy, om);
        // tau = rho nu (grad u + grad u^T) at each probe; Eq. 15 + Eq. 16 (per unit
        // length, then times the element length)
        const C mp = op.rho * nu, mm = om.rho * nu;
        const C txx = C(2) * (mp * op.dudx - mm * om.dudx);
        const C tyy = C(2) * (mp * op.dvdy - mm * om.dvdy);
        const C txy = mp * (op.dudy + op.dvdx) - mm * (om.dudy + om.dvdx);
        const C dp = op.p - om.p;
        const C nx = C(npx), ny = C(npy);
        const double len = (d.x * d.x + d.y * d.y) * rl;
        sm.ext[li] = make_double2((double)(-dp * nx + txx * nx + txy * ny) * len,
                                  (double)(-dp * ny + txy * nx + tyy * ny) * len);
    }
    if constexpr (F32) {
        if (P.ka != 0.0) {   // the enclosed area enters only Eq. 14's term, k_a (1 - A/A0)
            block_reduce<1, false>(area2f, sm.red);
            area2[0] = area2f[0];
        } else {
            __syncthreads();   // the staged terms and tractions, before the neighbours read them
        }
    } else {
        block_reduce<1, false>(area2, sm.red);
    }
    if (m == a.n) copy_halo_terms<F32>(sm, m, true);
    const double A = 0.5 * cluster_total(area2[0], arcs);
    if constexpr (F32) {
        // Eq. 14 factor k_a (1 - A/A0) p_ref / 2 from the exact difference A0 - A (no
        // double division on the narrow FP64 pipe)
        const float fa = (float)P.ka * ((float)(P.A0 - A) / (6.0f * (float)P.A0));
        const float hm = 0.5f / (float)P.m;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int li = kHalo + k, g = P.off + a.v0 + k;
            // the vertex's global inputs first, so that their latency overlaps the force terms
            const double2 Xm = nd.Xm1[g];
            const float2 xd = u_f(nd)[g];   // tentative velocity U of step 1 (Eq. 23)
            const float2 Fi = internal_force_f(sm, li - 1, li, li + 1, fa);
            const float2 e0 = ext_f(sm)[li], e1 = ext_f(sm)[li - 1];
            float2 Fe = make_float2(0.5f * (e0.x + e1.x), 0.5f * (e0.y + e1.y));
            if (nd.Fpp) {   // Eq. 27, part of the total force (step 7)
                const double2 f = nd.Fpp[g];
                Fe.x += (float)f.x;
                Fe.y += (float)f.y;
            }
            const double2 Xv = sm.X[li];
            // Eq. 23 as the increment X^{n+1} - X^n, and Eq. 24 as
            // 1.5 (X^{n+1} - X^n) - 0.5 (X^n - X^{n-1})
            const float ix = xd.x + hm * (Fi.x + Fe.x), iy = xd.y + hm * (Fi.y + Fe.y);
            const double dx = (double)ix, dy = (double)iy;
            // the last increment X^n - X^{n-1} as the exact double difference, the rest in
            // float (the velocity enters only the float force of the next spread)
            const float px = (float)(Xv.x - Xm.x), py = (float)(Xv.y - Xm.y);
            const double2 uvn = make_double2(1.5f * ix - 0.5f * px, 1.5f * iy - 0.5f * py);
            nd.uv[g] = uvn;
            nd.Xm1[g] = Xv;
            const double2 Xn = make_double2(Xv.x + dx, Xv.y + dy);
            nd.X[g] = Xn;
            if constexpr (NEXT) {
                // centre node of X^{n+1}: from the frame at X^n (offset d0 = c - X^n) and the
                // increment, in float; the offset itself as the exact double difference. A
                // non-finite or runaway position keeps the NaN mark of a position that is not
                // sane.
                MlsFrame f = reinterpret_cast<const MlsFrame*>(nd.mls)[g];
                const float px = ix - f.d0x, py = iy - f.d0y;   // X^{n+1} - c
                if (fabsf(px) < 1024.0f && fabsf(py) < 1024.0f) {   // false for NaN too
                    f.cx += (int)floorf(px + 0.5f);
                    f.cy += (int)floorf(py + 0.5f);
                    f.d0x = (float)((double)f.cx - Xn.x);
                    f.d0y = (float)((double)f.cy - Xn.y);
                } else {
                    f.d0x = __int_as_float(0x7fc00000);
                }
                reinterpret_cast<MlsFrame*>(nd.mls)[g] = f;
                // for the spread of the same CTA (only the float velocity enters its force)
                uv_next_f(sm)[li] = make_float2((float)uvn.x, (float)uvn.y);
                frame_c_f(sm)[li] = make_int2(f.cx, f.cy);
                frame_d_f(sm)[li] = make_float2(f.d0x, f.d0y);
                // the increment for the next step's element lengths (the slot's tentative
                // velocity is dead by now). The last forces are not stored: a fused update
                // never ends a call, and the update that does stores them.
                xd_f(sm)[li] = make_float2(ix, iy);
            } else {
                nd.Fint[g] = make_double2(Fi.x, Fi.y);
                nd.Fext[g] = make_double2(Fe.x, Fe.y);
            }
            nd.age[g] += 1;
        }
    } else {
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int li = kHalo + k, g = P.off + a.v0 + k;
            const double2 Fi = internal_force(sm, P, li - 1, li, li + 1, A);
            double2 Fe = 0.5 * (sm.ext[li] + sm.ext[li - 1]);
            if (nd.Fpp) Fe = Fe + nd.Fpp[g];   // Eq. 27, part of the total force (step 7)
            const double2 Xv = sm.X[li];
            const double2 Xm = nd.Xm1[g];
            const double2 xd = nd.U[g];
            const double hm = 0.5 / P.m;
            const double2 Xn = make_double2(Xv.x + xd.x + hm * (Fi.x + Fe.x), Xv.y + xd.y + hm * (Fi.y + Fe.y));
            nd.uv[g] = make_double2(1.5 * Xn.x - 2.0 * Xv.x + 0.5 * Xm.x, 1.5 * Xn.y - 2.0 * Xv.y + 0.5 * Xm.y);
            nd.Xm1[g] = Xv;
            nd.X[g] = Xn;
            nd.Fint[g] = Fi;
            nd.Fext[g] = Fe;
            nd.age[g] += 1;
        }
    }
    return ok;
}

template <typename S>
__global__ void __launch_bounds__(128, dyn_min_blocks<S>()) k_dyn_update(const S* __restrict__ dst, Lat L,
                                                    Nodes nd, int max_n, int arcs,
                                                    int tile_cells, int* reset_count, unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, arc_slots(max_n, arcs), kRedIB);
    if (blockIdx.x == 0 && threadIdx.x == 0 && reset_count) *reset_count = 0;
    CapsuleParams P;
    Arc a;
    if (!load_arc(nd, sm, max_n, arcs, true, P, a, status)) return;
    // a rigid particle's CTAs do no work here (k_rigid_update moves it); they take part in
    // the cluster's sums with nothing (a branch out would cost this kernel registers)
    const int m = P.rigid ? 0 : a.m;
    // vertices v0-1 .. v0+m: the ends of every element whose probes this CTA evaluates
    Tile<C> t = make_tile<C>(sm, kHalo - 1, m > 0 ? kHalo + m + 1 : kHalo - 1, 3, tile_cells, true, false);
    if (t.use) fill_moments<S>(t, dst, L, nullptr);
    __syncthreads();
    const bool ok = dyn_update<S>(dst, L, nd, P, a, sm, t, arcs, m);
    if (!ok) atomicOr(status, kStatSupport);
}

// Steps 7-8 of step n and steps 1-3 of step n+1 in one pass, for one CTA per capsule
// and no rigid particles (the host launches it only then). Both read the lattice state
// after step n's patch: the moments before any IB force. So the tile
// filled for the update at X^n also serves the interpolation and the spread at X^{n+1},
// whose supports lie inside the update's margin unless a vertex moved more than two
// lattice units in a step (flagged, as for any point that leaves its tile). The spread
// goes to the other force buffer and list (sp), whose counter the host has reset.
template <typename S>
__global__ void __launch_bounds__(128, dyn_min_blocks<S>()) k_dyn_update_spread(const S* __restrict__ dst, Lat L,
                                                                Nodes nd,
                                                                int max_n, int tile_cells, Spread sp,
                                                                unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, arc_slots(max_n, 1), kRedIB);
    CapsuleParams P;
    Arc a;
    if (!load_arc(nd, sm, max_n, 1, true, P, a, status)) return;
    Tile<C> t = make_tile<C>(sm, kHalo - 1, kHalo + a.m + 1, 3, tile_cells, true, true);
    if (t.use) {
        fill_moments<S>(t, dst, L, nullptr);
        zero_forces<C>(t);
    }
    __syncthreads();
    bool ok = dyn_update<S, true>(dst, L, nd, P, a, sm, t, 1, a.m);
    __syncthreads();   // every X^{n+1} is written (single precision: every increment staged)
    if constexpr (sizeof(C) == 4) {
        // the halo slots of the whole ring repeat its last and first vertex
        if (threadIdx.x == 0) {
            xd_f(sm)[kHalo - 1] = xd_f(sm)[kHalo + a.m - 1];
            xd_f(sm)[kHalo + a.m] = xd_f(sm)[kHalo];
        }
    } else {
        for (int li = threadIdx.x; li < a.m + 2 * kHalo; li += blockDim.x) sm.X[li] = nd.X[P.off + a.node(li)];
    }
    __syncthreads();
    ok &= dyn_spread<S, false, true>(dst, L, nd, P, a, sm, t, sp);
    __syncthreads();
    if (t.use) flush_forces<C>(t, L, sp, reinterpret_cast<int*>(sm.red));
    if (!ok) atomicOr(status, kStatSupport);
}

// Rigid particles after the fluid update (Section 2.3.1, Eq. 17-20): the outer probe of
// every element, the load summed over the particle (its CTAs form a cluster when its ring
// is split), then rigid_update. Capsules' CTAs return at once; launched only when the
// context holds rigid particles.
template <typename S>
__global__ void __launch_bounds__(128) k_rigid_update(const S* __restrict__ dst, Lat L,
                                                      Nodes nd, int max_n, int arcs,
                                                      int tile_cells, unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, arc_slots(max_n, arcs), kRedIB);
    CapsuleParams P;
    Arc a;
    if (!load_arc(nd, sm, max_n, arcs, true, P, a, status)) return;
    if (!P.rigid) return;   // uniform over the capsule's cluster
    const int m = a.m;
    Tile<C> t = make_tile<C>(sm, kHalo - 1, m > 0 ? kHalo + m + 1 : kHalo - 1, 3, tile_cells, true, false);
    if (t.use) fill_moments<S>(t, dst, L, nullptr);   // before any IB force, as the capsules' probes
    // the particle's state at n and n - 1, staged before the cluster barrier after which
    // the first CTA overwrites it
    __shared__ double body[12];
    if (threadIdx.x < 12)
        body[threadIdx.x] = threadIdx.x < 6 ? nd.rb[a.cap].body[threadIdx.x] : nd.rb[a.cap].prev[threadIdx.x - 6];
    __syncthreads();
    bool ok = true;
    double sums[3] = {0.0, 0.0, 0.0};   // F_x, F_y, M (Eq. 17-18)
    const C nu = C(L.nu);
    // own elements; a split ring also evaluates the element before its arc (for the
    // vertex shares of the first own vertex)
    const bool split = m > 0 && m < a.n;
    for (int k = threadIdx.x; k < (split ? m + 1 : m); k += blockDim.x) {
        const int li = k < m ? kHalo + k : kHalo - 1;
        const double2 Xv = sm.X[li], Xr = sm.X[li + 1];
        const double2 d = Xr - Xv;
        const double rl = rsqrt(d.x * d.x + d.y * d.y);
        const double npx = d.y * rl, npy = -d.x * rl;
        const double cx = 0.5 * (Xv.x + Xr.x), cy = 0.5 * (Xv.y + Xr.y);
        const double len = (d.x * d.x + d.y * d.y) * rl;
        InterpT<C> op;
        ok &= interp_at<S, true>(t, dst, L, nullptr, cx + 1.2 * npx, cy + 1.2 * npy, op);
        // Eq. 17: (tau+ . n+ - p+ n+) l_l of the outer fluid alone; Eq. 18: its moment
        // about c, lever arm to the element centroid. The reference pressure 1/3 adds
        // nothing over a closed ring (sum n_l l_l = 0, sum r_l x n_l l_l = 0) and is left
        // out, so that the load of a nearly balanced particle is not a small difference of
        // large single-precision terms.
        const C mp = op.rho * nu, nx = C(npx), ny = C(npy), pd = op.drho * C(1.0 / 3.0);
        const C txx = C(2) * mp * op.dudx, tyy = C(2) * mp * op.dvdy, txy = mp * (op.dudy + op.dvdx);
        const double fx = (double)(txx * nx + txy * ny - pd * nx) * len;
        const double fy = (double)(txy * nx + tyy * ny - pd * ny) * len;
        sm.ext[li] = make_double2(fx, fy);
        if (k < m) {
            sums[0] += fx;
            sums[1] += fy;
            sums[2] += (cx - body[0]) * fy - (cy - body[1]) * fx;
        }
    }
    if (nd.Fpp)   // Eq. 27 on the markers: part of the load and its moment
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const double2 f = nd.Fpp[P.off + a.v0 + k], X = sm.X[kHalo + k];
            sums[0] += f.x;
            sums[1] += f.y;
            sums[2] += (X.x - body[0]) * f.y - (X.y - body[1]) * f.x;
        }
    block_reduce<3, false>(sums, sm.red);   // also publishes the element forces
    if (m == a.n) {   // a whole ring: the element before the first vertex is the last one
        if (threadIdx.x == 0) sm.ext[kHalo - 1] = sm.ext[kHalo + m - 1];
        __syncthreads();
    }
    cluster_total<3>(sums, arcs);
    rigid_update(nd, P, a, sm, body, body + 6, sums);
    if (!ok) atomicOr(status, kStatSupport);
}

// ---------------------------------------------------------------------------------
// Kinematic IB (Section 2.4), steps i-iii: internal forces at X^n (Eq. 11, 13, 14) and
// their spread with c_v = 1. With arcs > 1 the capsule's CTAs form a cluster that sums
// the enclosed area. With float weights (single-precision storage) the membrane terms
// are in float too, as in the Dynamic kernels (positions, their differences and the
// strain's difference of squares stay double).
// ---------------------------------------------------------------------------------
// Steps i-iii on a staged arc whose force tile is zeroed (collective; a cluster over the
// capsule's CTAs when arcs > 1): the membrane terms, the enclosed area, the internal
// forces, the shape functions at the staged positions (stored for the node advance) and
// the spread. Returns false when a support left the channel or the tile.
template <typename C>
__device__ __forceinline__ bool kin_spread(const Lat& L, const Nodes& nd, const CapsuleParams& P, const Arc& a,
                                           const CapSmem& sm, Tile<C>& t, const Spread& sp, int arcs) {
    constexpr bool F32 = sizeof(C) == 4;
    const int m = a.m;
    double area2[1] = {0.0};
    float area2f[1] = {0.0f};
    // own slots, then (split ring) the halo slots kHalo-1 and kHalo+m
    const bool split = m > 0 && m < a.n;   // an arc without vertices has no tasks
    for (int k = threadIdx.x; k < (split ? m + 2 : m); k += blockDim.x) {
        const int li = k < m ? kHalo + k : (k == m ? kHalo - 1 : kHalo + m);
        if constexpr (F32) {
            vertex_terms_f(sm, P, nd, li - 1, li, li + 1, P.off + a.node(li));
            if (k < m) {
                const double2 Xv = sm.X[li];
                const float2 e = ring_f(sm)[li].e;
                area2f[0] += (float)(Xv.x - a.X0.x) * e.y - (float)(Xv.y - a.X0.y) * e.x;
            }
        } else {
            vertex_terms(sm, P, nd, li - 1, li, li + 1, P.off + a.node(li));
            if (k < m) area2[0] += area_term(a.X0, sm.X[li], sm.X[li + 1]);
        }
    }
    // the reductions also order the tile zeroing before the spread
    if constexpr (F32) {
        block_reduce<1, false>(area2f, sm.red);
        area2[0] = area2f[0];
    } else {
        block_reduce<1, false>(area2, sm.red);
    }
    if (m == a.n) copy_halo_terms<F32>(sm, m, false);
    const double A = 0.5 * cluster_total(area2[0], arcs);
    // Eq. 14 factor k_a (1 - A/A0) p_ref / 2 from the difference A0 - A (single precision)
    const float fa = F32 ? (float)P.ka * ((float)(P.A0 - A) / (6.0f * (float)P.A0)) : 0.0f;
    bool ok = true;
    // the spread in ring-hop order (see dyn_spread): fewer colliding shared-memory atomics
    const int hop = ring_hop(m);
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const int k = (int)((long long)j * hop % m);
        const int li = kHalo + k, g = P.off + a.v0 + k;
        double2 F;
        if constexpr (F32) {
            const float2 f = internal_force_f(sm, li - 1, li, li + 1, fa);
            F = make_double2(f.x, f.y);
        } else {
            F = internal_force(sm, P, li - 1, li, li + 1, A);
        }
        nd.Fint[g] = F;
        const double2 Fp = nd.Fpp ? nd.Fpp[g] : make_double2(0.0, 0.0);   // Eq. 27
        nd.Fext[g] = make_double2(0.0, 0.0);
        const MlsW<C> w = mls_setup<C>(L, sm.X[li].x, sm.X[li].y);
        store_mls<C>(nd.mls, g, w);
        ok &= spread_with<C>(w, t, L, sp, F.x + Fp.x, F.y + Fp.y, 1.0);
    }
    return ok;
}

// Kinematic IB (Section 2.4), steps i-iii: internal forces at X^n (Eq. 11, 13, 14) and
// their spread with c_v = 1. With arcs > 1 the capsule's CTAs form a cluster that sums
// the enclosed area. With float weights (single-precision storage) the membrane terms
// are in float too, as in the Dynamic kernels (positions, their differences and the
// strain's difference of squares stay double).
// ---------------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(128) k_kin_force_spread(Lat L, Nodes nd, int max_n, int arcs, int tile_cells,
                                                          Spread sp, unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, arc_slots(max_n, arcs), kRedIB);
    CapsuleParams P;
    Arc a;
    if (!load_arc(nd, sm, max_n, arcs, true, P, a, status)) return;
    Tile<C> t = make_tile<C>(sm, kHalo, kHalo + a.m, 1, tile_cells, false, true);
    if (t.use) zero_forces<C>(t);
    const bool ok = kin_spread<C>(L, nd, P, a, sm, t, sp, arcs);
    __syncthreads();
    if (t.use) flush_forces<C>(t, L, sp, reinterpret_cast<int*>(sm.red));
    if (!ok) atomicOr(status, kStatSupport);
}

// Kinematic IB steps vii-viii: xdot = I(u^{n+1}) at X^n with half the spread force,
// X^{n+1} = 2/3 (2 X^n - X^{n-1}/2 + xdot) (Eq. 25); forward Euler on a first step.
// Every CTA reads and writes only its own vertices.
template <typename S>
__global__ void __launch_bounds__(128, dyn_min_blocks<S>()) k_kin_advance(const S* __restrict__ dst, Lat L,
                                                     const double* __restrict__ fib, Nodes nd, int max_n, int arcs,
                                                     int tile_cells, int* reset_count, unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, arc_slots(max_n, arcs), kRedIB);
    if (blockIdx.x == 0 && threadIdx.x == 0 && reset_count) *reset_count = 0;
    CapsuleParams P;
    Arc a;
    if (!load_arc(nd, sm, max_n, arcs, false, P, a, status)) return;
    const int m = a.m;
    Tile<C> t = make_tile<C>(sm, kHalo, kHalo + m, 1, tile_cells, true, false);
    if (t.use) fill_moments<S>(t, dst, L, fib);
    __syncthreads();
    bool ok = true;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int g = P.off + a.v0 + k;
        const double2 Xv = sm.X[kHalo + k];
        InterpT<C> o;
        ok &= interp_with<S, false>(load_mls<C>(L, nd.mls, g), t, dst, L, fib, o);
        const double Ux = (double)o.ux, Uy = (double)o.uy;
        double2 Xn;
        if (nd.age[g] == 0) {
            Xn = make_double2(Xv.x + Ux, Xv.y + Uy);
        } else {
            const double2 Xm = nd.Xm1[g];
            Xn = make_double2((2.0 / 3.0) * (2.0 * Xv.x - 0.5 * Xm.x + Ux),
                              (2.0 / 3.0) * (2.0 * Xv.y - 0.5 * Xm.y + Uy));
        }
        nd.Xm1[g] = Xv;
        nd.X[g] = Xn;
        nd.uv[g] = make_double2(Ux, Uy);
        nd.age[g] += 1;
    }
    if (!ok) atomicOr(status, kStatSupport);
}

// Kinematic steps vii-viii of step n and steps i-iii of step n+1 in one pass, for one
// CTA per capsule without rigid particles or repulsion (the host launches it only then):
// the node advance at X^n as in k_kin_advance, X^{n+1} staged in place of X^n, then the
// spread at X^{n+1} into the next force buffer and list (sp, whose counter the host has
// reset). One tile serves both: the moments around X^n for the advance, the force
// accumulators for the spread, whose supports at X^{n+1} lie inside its margin of three
// nodes unless a vertex moved two lattice units in a step (flagged, as for any point that
// leaves its tile).
template <typename S>
__global__ void __launch_bounds__(128, dyn_min_blocks<S>()) k_kin_advance_spread(const S* __restrict__ dst, Lat L,
                                                                 const double* __restrict__ fib, Nodes nd,
                                                                 int max_n, int tile_cells, Spread sp,
                                                                 unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, arc_slots(max_n, 1), kRedIB);
    CapsuleParams P;
    Arc a;
    if (!load_arc(nd, sm, max_n, 1, true, P, a, status)) return;
    const int m = a.m;   // the whole ring
    Tile<C> t = make_tile<C>(sm, kHalo - 1, kHalo + m + 1, 3, tile_cells, true, true);
    if (t.use) {
        fill_moments<S>(t, dst, L, fib);
        zero_forces<C>(t);
    }
    __syncthreads();
    bool ok = true;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int li = kHalo + k, g = P.off + a.v0 + k;
        const double2 Xv = sm.X[li];
        InterpT<C> o;
        ok &= interp_with<S, false>(load_mls<C>(L, nd.mls, g), t, dst, L, fib, o);
        const double Ux = (double)o.ux, Uy = (double)o.uy;
        double2 Xn;
        if (nd.age[g] == 0) {
            Xn = make_double2(Xv.x + Ux, Xv.y + Uy);
        } else {
            const double2 Xm = nd.Xm1[g];
            Xn = make_double2((2.0 / 3.0) * (2.0 * Xv.x - 0.5 * Xm.x + Ux),
                              (2.0 / 3.0) * (2.0 * Xv.y - 0.5 * Xm.y + Uy));
        }
        nd.Xm1[g] = Xv;
        nd.X[g] = Xn;
        nd.uv[g] = make_double2(Ux, Uy);
        nd.age[g] += 1;
        sm.X[li] = Xn;   // only this thread reads the slot before the barrier
    }
    __syncthreads();
    // the halo slots repeat the ring's last and first vertices at X^{n+1}
    for (int h = threadIdx.x; h < 2 * kHalo; h += blockDim.x)
        sm.X[h < kHalo ? h : m + h] = sm.X[h < kHalo ? m + h : h];
    __syncthreads();
    ok &= kin_spread<C>(L, nd, P, a, sm, t, sp, 1);
    __syncthreads();
    if (t.use) flush_forces<C>(t, L, sp, reinterpret_cast<int*>(sm.red));
    if (!ok) atomicOr(status, kStatSupport);
}

// Observables of every capsule (Section 3.1-3.2): area, perimeter, Taylor D, centroid,
// swelling ratio, inclination, relative perimeter change.
__global__ void __launch_bounds__(128) k_observables(Nodes nd, int max_n, double* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    const CapsuleParams P = nd.caps[blockIdx.x];
    const int n = P.n, off = P.off;
    if (n < 3 || off < 0 || off + n > nd.count) return;
    const double2 X0 = nd.X[off];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};  // 2A, sx, sy, sxx, syy, sxy, perimeter
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 a = nd.X[off + i] - X0, b = nd.X[off + (i + 1 == n ? 0 : i + 1)] - X0;
        const double c = a.x * b.y - b.x * a.y;
        s[0] += c;
        s[1] += (a.x + b.x) * c;
        s[2] += (a.y + b.y) * c;
        s[3] += (a.x * a.x + a.x * b.x + b.x * b.x) * c;
        s[4] += (a.y * a.y + a.y * b.y + b.y * b.y) * c;
        s[5] += (a.x * b.y + 2.0 * a.x * a.y + 2.0 * b.x * b.y + b.x * a.y) * c;
        s[6] += sqrt((b.x - a.x) * (b.x - a.x) + (b.y - a.y) * (b.y - a.y));
    }
    block_reduce<7, false>(s, sm.red);
    if (threadIdx.x == 0) {
        const double A = 0.5 * s[0];
        const double cx = s[1] / (6.0 * A), cy = s[2] / (6.0 * A);
        const double Ixx = s[3] / 12.0 - A * cx * cx;
        const double Iyy = s[4] / 12.0 - A * cy * cy;
        const double Ixy = s[5] / 24.0 - A * cx * cy;
        const double mid = 0.5 * (Ixx + Iyy);
        const double dd = sqrt(0.25 * (Ixx - Iyy) * (Ixx - Iyy) + Ixy * Ixy);
        const double lmax = (mid + dd) / A, lmin = (mid - dd) / A;
        const double a = 2.0 * sqrt(lmax), b = 2.0 * sqrt(lmin > 0.0 ? lmin : 0.0);
        const double Pm = s[6];
        double* o = out + 8 * blockIdx.x;
        o[0] = A;
        o[1] = Pm;
        o[2] = (a - b) / (a + b);
        o[3] = cx + X0.x;
        o[4] = cy + X0.y;
        o[5] = A / (Pm * Pm / (4.0 * 3.14159265358979323846));
        o[6] = 0.5 * atan2(2.0 * Ixy, Ixx - Iyy);
        o[7] = (Pm - P.P0) / P.P0;
    }
}

// MLS interpolation (Eq. 8) with gradient at arbitrary points.
template <typename S>
__global__ void k_interp_points(const S* __restrict__ src, Lat L, const double* __restrict__ fib,
                                const double2* __restrict__ pts, int n, double* __restrict__ out,
                                unsigned* status) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    InterpT<typename St<S>::C> o;
    const bool ok = mls_interp<S, true>(src, L, fib, pts[m].x, pts[m].y, o);
    double* r = out + 8 * (long long)m;
    r[0] = o.ux; r[1] = o.uy; r[2] = o.rho; r[3] = o.p;
    r[4] = o.dudx; r[5] = o.dudy; r[6] = o.dvdx; r[7] = o.dvdy;
    if (!ok) atomicOr(status, kStatSupport);
}

// ---------------------------------------------------------------------------------
// Host launchers. `tile_cells` is the per-capsule tile budget chosen by the host from
// the capsules' reference extent (tile_budget()).
// ---------------------------------------------------------------------------------
static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// keep well clear of the 227 KB opt-in limit (static shared variables come on top)
constexpr size_t kSmemLimit = 200 * 1024;

template <typename C>
static size_t tile_bytes(int cells, bool moments, bool forces) {
    // the flush scratch (one int per cell) lives in the moment arrays or behind the
    // force accumulators
    const size_t m = moments ? 3 * sizeof(C) : 0;
    const size_t f = forces ? 2 * sizeof(C) + (moments ? 0 : sizeof(int)) : 0;
    return (size_t)cells * (m + f);
}

template <typename C>
static size_t smem_bytes(int slots, int cells, bool moments, bool forces) {
    return ring_smem_bytes(slots, kRedIB) + tile_bytes<C>(cells, moments, forces);
}

int tile_budget(int slots, double extent, bool tight) {
    // a square of side `extent` plus the probes and supports (3 nodes each side); for a
    // whole ring 1.5 x that, room for any rotation and for deformation
    const double side = extent + 8.0;
    long long cells = (long long)((tight ? 1.0 : 1.15) * side * side);
    if (cells < 256) cells = 256;
    const size_t free_b = kSmemLimit - ring_smem_bytes(slots, kRedIB);
    const long long cap = (long long)(free_b / (3 * sizeof(double) + 2 * sizeof(double)));
    if (cells > cap) cells = cap;
    return (int)cells;
}

// The limits are per kernel and process-wide: raise them, never lower them, so that
// contexts of different ring sizes can run side by side.
void set_capsule_smem_limits(int slots, int cells) {
    static std::mutex mu;
    static std::map<const void*, size_t> set;
    std::lock_guard<std::mutex> lock(mu);
    auto raise = [&](const void* k, size_t bytes) {
        size_t& cur = set[k];
        if (bytes <= cur) return;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess) cur = bytes;
    };
#define LBMIB_SMEM(K, C, M, F) raise((const void*)K, smem_bytes<C>(slots, cells, M, F))
    LBMIB_SMEM((k_dyn_force_spread<double, false>), double, true, true);
    LBMIB_SMEM((k_dyn_force_spread<float, false>), float, true, true);
    LBMIB_SMEM((k_dyn_force_spread<__half, false>), float, true, true);
    LBMIB_SMEM((k_dyn_force_spread<double, true>), double, true, true);
    LBMIB_SMEM((k_dyn_force_spread<float, true>), float, true, true);
    LBMIB_SMEM((k_dyn_force_spread<__half, true>), float, true, true);
    LBMIB_SMEM(k_rigid_update<double>, double, true, false);
    LBMIB_SMEM(k_rigid_update<float>, float, true, false);
    LBMIB_SMEM(k_rigid_update<__half>, float, true, false);
    LBMIB_SMEM(k_dyn_update<double>, double, true, false);
    LBMIB_SMEM(k_dyn_update<float>, float, true, false);
    LBMIB_SMEM(k_dyn_update<__half>, float, true, false);
    LBMIB_SMEM((k_dyn_force_spread<f32w, false>), double, true, true);
    LBMIB_SMEM((k_dyn_force_spread<f16w, false>), double, true, true);
    LBMIB_SMEM((k_dyn_force_spread<f32w, true>), double, true, true);
    LBMIB_SMEM((k_dyn_force_spread<f16w, true>), double, true, true);
    LBMIB_SMEM(k_rigid_update<f32w>, double, true, false);
    LBMIB_SMEM(k_rigid_update<f16w>, double, true, false);
    LBMIB_SMEM(k_dyn_update<f32w>, double, true, false);
    LBMIB_SMEM(k_dyn_update<f16w>, double, true, false);
    LBMIB_SMEM(k_dyn_update_spread<f32w>, double, true, true);
    LBMIB_SMEM(k_dyn_update_spread<f16w>, double, true, true);
    LBMIB_SMEM(k_kin_advance<f32w>, double, true, false);
    LBMIB_SMEM(k_kin_advance<f16w>, double, true, false);
    LBMIB_SMEM(k_dyn_update_spread<double>, double, true, true);
    LBMIB_SMEM(k_dyn_update_spread<float>, float, true, true);
    LBMIB_SMEM(k_dyn_update_spread<__half>, float, true, true);
    LBMIB_SMEM(k_kin_advance_spread<double>, double, true, true);
    LBMIB_SMEM(k_kin_advance_spread<float>, float, true, true);
    LBMIB_SMEM(k_kin_advance_spread<__half>, float, true, true);
    LBMIB_SMEM(k_kin_advance_spread<f32w>, double, true, true);
    LBMIB_SMEM(k_kin_advance_spread<f16w>, double, true, true);
    LBMIB_SMEM(k_kin_advance<double>, double, true, false);
    LBMIB_SMEM(k_kin_advance<float>, float, true, false);
    LBMIB_SMEM(k_kin_advance<__half>, float, true, false);
    LBMIB_SMEM(k_kin_force_spread<double>, double, false, true);
    LBMIB_SMEM(k_kin_force_spread<float>, float, false, true);
#undef LBMIB_SMEM
}

// Launch a capsule kernel over ncaps x arcs CTAs of 128 threads; with `cluster`, each
// capsule's arcs form one thread-block cluster.
template <typename... P, typename... A>
static void launch_arcs(void (*k)(P...), int ncaps, int arcs, bool cluster, size_t smem, cudaStream_t s,
                        A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ncaps * (unsigned)arcs);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    if (cluster && arcs > 1) {
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)arcs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

template <typename S>
void launch_dyn_force_spread(const void* src, const Lat& L, Nodes nd, int ncaps, int max_n,
                             int arcs, int cells, bool rigid, Spread sp, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    const size_t sh = smem_bytes<C>(arc_slots(max_n, arcs), cells, true, true);
    if (rigid)
        launch_arcs(k_dyn_force_spread<S, true>, ncaps, arcs, false, sh, s, (const S*)src, L, nd, max_n,
                    arcs, cells, sp, status);
    else
        launch_arcs(k_dyn_force_spread<S, false>, ncaps, arcs, false, sh, s, (const S*)src, L, nd, max_n,
                    arcs, cells, sp, status);
}

template <typename S>
void launch_dyn_update(const void* dst, const Lat& L, Nodes nd, int ncaps, int max_n,
                       int arcs, int cells, bool rigid, int* reset_count, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    const size_t sh = smem_bytes<C>(arc_slots(max_n, arcs), cells, true, false);
    launch_arcs(k_dyn_update<S>, ncaps, arcs, true, sh, s, (const S*)dst, L, nd, max_n, arcs, cells,
                reset_count, status);
    if (rigid)
        launch_arcs(k_rigid_update<S>, ncaps, arcs, true, sh, s, (const S*)dst, L, nd, max_n, arcs, cells,
                    status);
}

template <typename S>
void launch_dyn_update_spread(const void* dst, const Lat& L, Nodes nd, int ncaps, int max_n,
                              int cells, Spread sp_next, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    const size_t sh = smem_bytes<C>(arc_slots(max_n, 1), cells, true, true);
    launch_arcs(k_dyn_update_spread<S>, ncaps, 1, false, sh, s, (const S*)dst, L, nd, max_n, cells, sp_next,
                status);
}

void launch_kin_force_spread(const Lat& L, Nodes nd, int ncaps, int max_n, int arcs, int cells, Spread sp,
                             unsigned* status, bool fp64_weights, cudaStream_t s) {
    // double MLS weights when the populations are double, float otherwise
    const int slots = arc_slots(max_n, arcs);
    if (fp64_weights)
        launch_arcs(k_kin_force_spread<double>, ncaps, arcs, true, smem_bytes<double>(slots, cells, false, true), s,
                    L, nd, max_n, arcs, cells, sp, status);
    else
        launch_arcs(k_kin_force_spread<float>, ncaps, arcs, true, smem_bytes<float>(slots, cells, false, true), s,
                    L, nd, max_n, arcs, cells, sp, status);
}

template <typename S>
void launch_kin_advance(const void* dst, const Lat& L, const double* fib_cur, Nodes nd, int ncaps, int max_n,
                        int arcs, int cells, int* reset_count, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    launch_arcs(k_kin_advance<S>, ncaps, arcs, false, smem_bytes<C>(arc_slots(max_n, arcs), cells, true, false), s,
                (const S*)dst, L, fib_cur, nd, max_n, arcs, cells, reset_count, status);
}

template <typename S>
void launch_kin_advance_spread(const void* dst, const Lat& L, const double* fib_cur, Nodes nd, int ncaps, int max_n,
                               int cells, Spread sp_next, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    launch_arcs(k_kin_advance_spread<S>, ncaps, 1, false, smem_bytes<C>(arc_slots(max_n, 1), cells, true, true), s,
                (const S*)dst, L, fib_cur, nd, max_n, cells, sp_next, status);
}

void launch_observables(Nodes nd, int ncaps, int max_n, double* out, cudaStream_t s) {
    // set here rather than with the other limits: contexts and batches of different ring
    // sizes share this kernel
    cudaFuncSetAttribute(k_observables, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_smem_bytes(max_n));
    k_observables<<<ncaps, 128, ring_smem_bytes(max_n), s>>>(nd, max_n, out);
}

template <typename S>
void launch_interp_points(const void* src, const Lat& L, const double* fib, const double2* pts, int n,
                          double* out, unsigned* status, cudaStream_t s) {
    k_interp_points<S><<<nblk(n, 128), 128, 0, s>>>((const S*)src, L, fib, pts, n, out, status);
}

#define LBMIB_INSTANTIATE_IB(S)                                                                              \
    template void launch_dyn_force_spread<S>(const void*, const Lat&, Nodes, int, int, int, int, bool,       \
                                             Spread, unsigned*, cudaStream_t);                               \
    template void launch_dyn_update<S>(const void*, const Lat&, Nodes, int, int, int, int, bool, int*,       \
                                       unsigned*, cudaStream_t);                                             \
    template void launch_dyn_update_spread<S>(const void*, const Lat&, Nodes, int, int, int, Spread,         \
                                              unsigned*, cudaStream_t);                                      \
    template void launch_kin_advance<S>(const void*, const Lat&, const double*, Nodes, int, int, int, int,   \
                                        int*, unsigned*, cudaStream_t);                                      \
    template void launch_kin_advance_spread<S>(const void*, const Lat&, const double*, Nodes, int, int, int,  \
                                               Spread, unsigned*, cudaStream_t);                             \
    template void launch_interp_points<S>(const void*, const Lat&, const double*, const double2*, int,       \
                                          double*, unsigned*, cudaStream_t);

LBMIB_INSTANTIATE_IB(double)
LBMIB_INSTANTIATE_IB(float)
LBMIB_INSTANTIATE_IB(__half)
LBMIB_INSTANTIATE_IB(f32w)
LBMIB_INSTANTIATE_IB(f16w)

}  // namespace lbmib
