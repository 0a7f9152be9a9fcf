// Device helpers shared by the immersed-boundary kernels (ib.cu) and the batched
// persistent kernel (batch.cu): the shared-memory view of one capsule, block
// reductions, the capsule tile, and the membrane force terms (Eq. 10-14).
#pragma once

#include "lbmib_kernels.cuh"

namespace lbmib {

// Shared-memory view of one capsule (sized by the largest ring of the launch).
struct CapSmem {
    double2* X;     // vertex positions
    double2* ext;   // external force of element v (v -> v+1), Eq. 15-16
    double2* xd;    // interpolated velocity at vertex v
    double* sst;    // stretch factor of element v: -k_s (l - l_0) / l  (Eq. 11)
    double* bs;     // k_b sin(theta_v - theta_v0) at vertex v            (Eq. 13)
    double2* bdl;   // d(theta_v)/dX_{v-1}
    double2* bdr;   // d(theta_v)/dX_{v+1}
    double* red;    // reduction scratch (8 doubles per warp of the block)
    unsigned char* tile;  // moment / force tile
};

// red_doubles: the reduction scratch, 8 doubles per warp of the launch (the default
// covers blocks of up to 1024 threads)
inline size_t ring_smem_bytes(int max_n, int red_doubles = 32 * 8) {
    return (size_t)max_n * (5 * sizeof(double2) + 2 * sizeof(double)) + (size_t)red_doubles * sizeof(double);
}

__device__ __forceinline__ CapSmem carve(unsigned char* base, int max_n, int red_doubles = 32 * 8) {
    CapSmem s;
    s.X = reinterpret_cast<double2*>(base);
    s.ext = s.X + max_n;
    s.xd = s.ext + max_n;
    s.bdl = s.xd + max_n;
    s.bdr = s.bdl + max_n;
    s.sst = reinterpret_cast<double*>(s.bdr + max_n);
    s.bs = s.sst + max_n;
    s.red = s.bs + max_n;
    s.tile = reinterpret_cast<unsigned char*>(s.red + red_doubles);
    return s;
}

// Reduction of K doubles or floats over the block (blockDim.x a multiple of 32, <= 1024);
// MIN selects minimum instead of sum. Every thread receives the results. `red_` is the
// block's double scratch (8 doubles per warp).
template <int K, bool MIN, typename T>
__device__ void block_reduce(T (&v)[K], double* red_) {
    T* red = reinterpret_cast<T*>(red_);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++)
        for (int o = 16; o > 0; o >>= 1) {
            const T t = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = MIN ? fmin(v[k], t) : v[k] + t;
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) red[warp * K + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
        T t = red[k];
        for (int w = 1; w < nw; w++) t = MIN ? fmin(t, red[w * K + k]) : t + red[w * K + k];
        v[k] = t;
    }
    __syncthreads();
}

__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// ---------------------------------------------------------------------------------
// Capsule tile: lattice moments (and, for the spread, force accumulators) of every node
// in the bounding box of the ring widened by `margin` nodes.
// ---------------------------------------------------------------------------------
template <typename C>
struct Tile {
    int x0, y0, w, h;   // origin (unwrapped lattice coordinates) and extent
    bool use;           // the box fits the tile budget
    C* drho;
    C* ux;
    C* uy;
    C* fx;              // force accumulators (compute type)
    C* fy;
    int* cells;         // scratch for the flush (aliases the moment arrays)

    __device__ __forceinline__ int index(int x, int y) const { return (y - y0) * w + (x - x0); }
    // the 3x3 support centred on (cx, cy) lies inside the tile
    __device__ __forceinline__ bool holds(int cx, int cy) const {
        return use && cx - 1 >= x0 && cx + 1 < x0 + w && cy - 1 >= y0 && cy + 1 < y0 + h;
    }
};

// Bounding box of the staged slots [lo, hi) and the tile layout (no tile for an empty
// range). Collective (all threads). Only the floors of the extreme coordinates matter,
// so the box is reduced in float (off the narrow FP64 pipe): every coordinate is rounded
// down to float, which keeps its floor while |X| < 2^24 (every integer up to there is a
// float), and floor is monotone, so the floors of the float minima and maxima are those of
// the double ones. A box reaching beyond 2^24 (a runaway capsule) takes no tile.
template <typename C>
__device__ Tile<C> make_tile(const CapSmem& sm, int lo, int hi, int margin, int tile_cells, bool moments,
                             bool forces) {
    constexpr float kBig = 3.0e38f, kLimit = 16777216.0f;
    float r[4] = {kBig, kBig, kBig, kBig};  // min x, min y, -max x, -max y
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const double2 X = sm.X[v];
        const float x = __double2float_rd(X.x), y = __double2float_rd(X.y);   // NaN: ignored by fminf
        r[0] = fminf(r[0], x);
        r[1] = fminf(r[1], y);
        r[2] = fminf(r[2], -x);
        r[3] = fminf(r[3], -y);
    }
    block_reduce<4, true>(r, sm.red);
    Tile<C> t;
    const bool sane = fabsf(r[0]) < kLimit && fabsf(r[1]) < kLimit && fabsf(r[2]) < kLimit && fabsf(r[3]) < kLimit;
    t.x0 = sane ? (int)floorf(r[0]) - margin : 0;
    t.y0 = sane ? (int)floorf(r[1]) - margin : 0;
    const long long w = sane ? (long long)floorf(-r[2]) + 1 + margin - t.x0 + 1 : 1LL << 30;
    const long long h = sane ? (long long)floorf(-r[3]) + 1 + margin - t.y0 + 1 : 1LL << 30;
    t.use = sane && w * h <= tile_cells;
    t.w = t.use ? (int)w : 0;
    t.h = t.use ? (int)h : 0;
    unsigned char* p = sm.tile;
    t.drho = t.ux = t.uy = nullptr;
    t.fx = t.fy = nullptr;
    t.cells = reinterpret_cast<int*>(p);
    if (forces) {
        t.fx = reinterpret_cast<C*>(p);
        t.fy = t.fx + tile_cells;
        p += 2 * sizeof(C) * (size_t)tile_cells;
        t.cells = reinterpret_cast<int*>(p);   // behind the accumulators
    }
    if (moments) {
        t.drho = reinterpret_cast<C*>(p);
        t.ux = t.drho + tile_cells;
        t.uy = t.ux + tile_cells;
    }
    return t;
}

// Zero the force accumulators of a tile (collective; callers order it before use).
template <typename C>
__device__ void zero_forces(Tile<C>& t) {
    const int cells = t.w * t.h;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        t.fx[k] = C(0);
        t.fy[k] = C(0);
    }
}

// Stretch factor of element v and bending terms of vertex v (Eq. 11, 13) into the
// staged slots: vl, v, vr are the slots of X_{v-1}, X_v, X_{v+1}; g is v's index in
// the node arrays.
__device__ __forceinline__ void vertex_terms(const CapSmem& sm, const CapsuleParams& P, const Nodes& nd, int vl,
                                             int v, int vr, int g) {
    const double2 Xv = sm.X[v], Xr = sm.X[vr], Xl = sm.X[vl];
    const double2 a = Xv - Xl, b = Xr - Xv;   // incoming edge, outgoing edge (element v)
    const double a2 = a.x * a.x + a.y * a.y, b2 = b.x * b.x + b.y * b.y;
    const double ra = rsqrt(a2), rb = rsqrt(b2);   // 1/|a|, 1/|b|
    // Eq. 11: element v joins v and v+1, length |b|
    sm.sst[v] = -P.ks * (b2 * rb - nd.L0[g]) * rb;
    // Eq. 13 as F = -k_b sin(theta - theta_0) d(theta)/dX with theta the signed turning
    // angle at v; sin(theta - theta_0) from the cross and dot products and theta_0's
    // stored cosine and sine.
    const double cr = a.x * b.y - a.y * b.x, dt = a.x * b.x + a.y * b.y;
    const double sdiff = (cr * nd.c0[g] - dt * nd.s0[g]) * (ra * rb);
    sm.bs[v] = P.kb * sdiff;
    const double ia2 = ra * ra, ib2 = rb * rb;
    sm.bdl[v] = make_double2(-a.y * ia2, a.x * ia2);
    sm.bdr[v] = make_double2(-b.y * ib2, b.x * ib2);
}

// ---------------------------------------------------------------------------------
// Single-precision membrane terms (FP32 and FP16 storage). Positions stay double; the
// edge vectors are formed as double differences and then held in float, and the
// stretch strain uses the difference of squares |b|^2 - L0^2 in double, so that the
// strain keeps its relative precision however close |b| is to L0. The terms of a staged
// slot live in the storage of the double bending derivatives (32 bytes per slot, bdl
// and bdr being adjacent arrays), the element tractions and vertex velocities in the
// first half of their double slots.
// ---------------------------------------------------------------------------------
struct RingF {
    float sst, bs;    // stretch factor of element v, k_b sin(theta_v - theta_v0)
    float2 bdl, bdr;  // d(theta_v)/dX_{v-1}, d(theta_v)/dX_{v+1}
    float2 e;         // element vector X_{v+1} - X_v
};
static_assert(sizeof(RingF) == 2 * sizeof(double2), "a RingF slot spans one bdl and one bdr slot");

__device__ __forceinline__ RingF* ring_f(const CapSmem& sm) { return reinterpret_cast<RingF*>(sm.bdl); }
__device__ __forceinline__ float2* ext_f(const CapSmem& sm) { return reinterpret_cast<float2*>(sm.ext); }
__device__ __forceinline__ float2* xd_f(const CapSmem& sm) { return reinterpret_cast<float2*>(sm.xd); }
__device__ __forceinline__ float* len_f(const CapSmem& sm) { return reinterpret_cast<float*>(sm.sst); }
// the Dynamic scheme's per-vertex U as float in single precision (the first half of its slots)
__device__ __forceinline__ float2* u_f(const Nodes& nd) { return reinterpret_cast<float2*>(nd.U); }
// What the fused single-precision update hands to the next step's spread in the same CTA
// (so that the spread reloads nothing from global memory): the new vertex velocity in
// float in the double slots of sm.bs, which the float terms leave unused, and the new
// support frame split over the unused second halves of the ext and xd arrays.
__device__ __forceinline__ float2* uv_next_f(const CapSmem& sm) { return reinterpret_cast<float2*>(sm.bs); }
__device__ __forceinline__ int2* frame_c_f(const CapSmem& sm) {
    return reinterpret_cast<int2*>(sm.ext) + (sm.xd - sm.ext);
}
__device__ __forceinline__ float2* frame_d_f(const CapSmem& sm) {
    return reinterpret_cast<float2*>(sm.xd) + (sm.bdl - sm.xd);
}

// vertex_terms in single precision (the same Eq. 11 and Eq. 13 terms).
__device__ __forceinline__ void vertex_terms_f(const CapSmem& sm, const CapsuleParams& P, const Nodes& nd, int vl,
                                               int v, int vr, int g) {
    const double2 Xv = sm.X[v], Xr = sm.X[vr], Xl = sm.X[vl];
    const double2 ad = Xv - Xl, bd = Xr - Xv;   // incoming edge, outgoing edge (element v)
    const double L0 = nd.L0[g];
    const double b2d = bd.x * bd.x + bd.y * bd.y;
    const float dsq = (float)fma(-L0, L0, b2d);   // |b|^2 - L0^2
    const float2 a = make_float2((float)ad.x, (float)ad.y), b = make_float2((float)bd.x, (float)bd.y);
    const float a2 = a.x * a.x + a.y * a.y, b2 = (float)b2d;
    const float ra = rsqrtf(a2), rb = rsqrtf(b2);
    const float lb = b2 * rb;
    RingF& o = ring_f(sm)[v];
    // Eq. 11: -k_s (|b| - L0) / |b| with |b| - L0 = (|b|^2 - L0^2) / (|b| + L0)
    o.sst = -(float)P.ks * dsq / ((lb + (float)L0) * lb);
    // Eq. 13: k_b sin(theta - theta_0) from the cross and dot products
    const float cr = a.x * b.y - a.y * b.x, dt = a.x * b.x + a.y * b.y;
    o.bs = (float)P.kb * ((cr * (float)nd.c0[g] - dt * (float)nd.s0[g]) * (ra * rb));
    const float ia2 = ra * ra, ib2 = rb * rb;
    o.bdl = make_float2(-a.y * ia2, a.x * ia2);
    o.bdr = make_float2(-b.y * ib2, b.x * ib2);
    o.e = b;
}

// internal_force in single precision from the float terms of slots vl, v, vr; fa is the
// Eq. 14 factor k_a (1 - A/A0) p_ref / 2.
__device__ __forceinline__ float2 internal_force_f(const CapSmem& sm, int vl, int v, int vr, float fa) {
    const RingF* R = ring_f(sm);
    const RingF c = R[v], l = R[vl];
    const float bsr = R[vr].bs;
    const float2 bdlr = R[vr].bdl;
    // stretch: element v (this vertex first, X_v - X_{v+1} = -e_v) and element v-1 (this
    // vertex second, X_{v-1} - X_v = -e_{v-1}); bending: own angle, as left neighbour of
    // v+1, as right neighbour of v-1; area: (dy, -dx) of both elements, half each
    float fx = -c.sst * c.e.x + l.sst * l.e.x + c.bs * (c.bdl.x + c.bdr.x) - bsr * bdlr.x - l.bs * l.bdr.x;
    float fy = -c.sst * c.e.y + l.sst * l.e.y + c.bs * (c.bdl.y + c.bdr.y) - bsr * bdlr.y - l.bs * l.bdr.y;
    fx += fa * (c.e.y + l.e.y);
    fy -= fa * (c.e.x + l.e.x);
    return make_float2(fx, fy);
}

// Element v's contribution to twice the enclosed area (Green's theorem about X_0).
__device__ __forceinline__ double area_term(double2 X0, double2 Xv, double2 Xr) {
    return (Xv.x - X0.x) * (Xr.y - X0.y) - (Xr.x - X0.x) * (Xv.y - X0.y);
}

// Per-element stretch factor and per-vertex bending terms of vertex/element v of a
// whole staged ring, and this vertex's contribution to twice the enclosed area.
__device__ __forceinline__ double ring_terms(const CapSmem& sm, const CapsuleParams& P, const Nodes& nd, int v) {
    const int n = P.n;
    const int vr = v + 1 == n ? 0 : v + 1;
    vertex_terms(sm, P, nd, v == 0 ? n - 1 : v - 1, v, vr, P.off + v);
    return area_term(sm.X[0], sm.X[v], sm.X[vr]);
}

// Internal force on the vertex in slot v (Eq. 22: stretch + bending + area) from the
// staged terms of slots vl, v, vr (its neighbours) and the enclosed area A.
__device__ __forceinline__ double2 internal_force(const CapSmem& sm, const CapsuleParams& P, int vl, int v, int vr,
                                                  double A) {
    const double2 Xv = sm.X[v], Xl = sm.X[vl], Xr = sm.X[vr];
    double2 F = sm.sst[v] * (Xv - Xr);           // element v, this vertex first
    F = F + (-sm.sst[vl]) * (Xl - Xv);           // element v-1, this vertex second
    F = F + sm.bs[v] * (sm.bdl[v] + sm.bdr[v]);  // own bending angle
    F = F + (-sm.bs[vr]) * sm.bdl[vr];           // as left neighbour of v+1
    F = F + (-sm.bs[vl]) * sm.bdr[vl];           // as right neighbour of v-1
    // Eq. 14: F^a_l = k_a (1 - A/A0) p_ref (dy, -dx) for element l, half to each end
    const double fa = P.ka * (1.0 - A / P.A0) * (1.0 / 3.0) * 0.5;
    const double2 dr = Xr - Xv, dl = Xv - Xl;
    F.x += fa * (dr.y + dl.y);
    F.y -= fa * (dr.x + dl.x);
    return F;
}

// Internal force on vertex v of a whole staged ring.
__device__ __forceinline__ double2 node_internal_force(const CapSmem& sm, const CapsuleParams& P, int v, double A) {
    const int n = P.n;
    return internal_force(sm, P, v == 0 ? n - 1 : v - 1, v, v + 1 == n ? 0 : v + 1, A);
}

}  // namespace lbmib
