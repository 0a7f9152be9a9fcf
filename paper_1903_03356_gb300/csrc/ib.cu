// Immersed-boundary kernels: MLS interpolation and spreading (Eq. 8-9, Section 2.3
// step 3, Section 2.4 step iii), membrane forces (Eq. 10-14), hydrodynamic tractions
// (Eq. 15-16), and the node updates of the Dynamic (Eq. 21-24) and Kinematic (Eq. 25)
// schemes. Coclite et al., arXiv:1903.03356.
//
// Every kernel here runs one CTA per capsule. The CTA stages its ring in shared memory,
// takes the bounding box of the ring (plus the reach of the supports, and of the
// probes when it needs them) and fills a shared tile with the lattice moments of every
// node in the box once (nine pulls per node). Node and probe interpolations then read
// that tile instead of re-gathering 81 populations each, and the spread accumulates
// into a shared force tile that is flushed once per touched node (one global atomic
// per node instead of one per marker and support point). A capsule whose box does not
// fit the tile budget takes the same path with global pulls and global atomics.
// Positions, velocities, forces, reference lengths and the MLS reciprocals are double
// in every storage mode; in FP32/FP16 modes the weights and weighted sums are float.
#include "ring.cuh"

namespace lbmib {

size_t capsule_smem_bytes(int max_n) { return ring_smem_bytes(max_n); }

// Fill the moment tile from the populations (nine pulls per node, row by row).
template <typename S>
__device__ void fill_moments(Tile<typename St<S>::C>& t, const S* __restrict__ src, const Lat& L,
                             const double* __restrict__ fib) {
    using C = typename St<S>::C;
    const int cells = t.w * t.h;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        const int j = k / t.w, i = k - j * t.w;
        const Mom<C> m = node_moments<S>(src, L, fib, wrapi(t.x0 + i, L.nx), support_row(L, t.y0 + j));
        t.drho[k] = m.drho;
        t.ux[k] = m.ux;
        t.uy[k] = m.uy;
    }
}

__device__ __forceinline__ void touch(const Spread& sp, int cell, int stamp) {
    if (atomicExch(&sp.mark[cell], stamp) != stamp) {
        const int p = atomicAdd(sp.count, 1);
        if (p < sp.capacity) sp.list[p] = cell;
        else atomicOr(sp.status, kStatList);
    }
}

// Add the force tile to the lattice force field and record the touched nodes. The
// nodes new to this step's list are collected in shared memory first and appended with
// one global reservation per capsule, so that the list counter is not a hot spot.
// Collective (all threads); the moment arrays are dead by now and hold the scratch.
template <typename C>
__device__ void flush_forces(const Tile<C>& t, const Lat& L, const Spread& sp, int stamp, int* s_count) {
    const long long N = (long long)L.nx * L.ny;
    const int cells = t.w * t.h;
    if (threadIdx.x == 0) *s_count = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        const double fx = (double)t.fx[k], fy = (double)t.fy[k];
        if (fx == 0.0 && fy == 0.0) continue;
        const int j = k / t.w, i = k - j * t.w;
        const int cell = support_row(L, t.y0 + j) * L.nx + wrapi(t.x0 + i, L.nx);
        atomicAdd(sp.fib + cell, fx);
        atomicAdd(sp.fib + N + cell, fy);
        if (atomicExch(&sp.mark[cell], stamp) != stamp) t.cells[atomicAdd(s_count, 1)] = cell;
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
__device__ __forceinline__ bool spread_with(const MlsW<C>& m, Tile<C>& t, const Lat& L, const Spread& sp, int stamp,
                                            double Fx, double Fy, double c) {
    const long long N = (long long)L.nx * L.ny;
    const bool in_tile = t.holds(m.cx, m.cy);
    const C cFx = C(c * Fx), cFy = C(c * Fy);
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
                const double w = c * (double)phi;
                const int cell = support_row(L, m.cy + b - 1) * L.nx + wrapi(m.cx + a - 1, L.nx);
                atomicAdd(sp.fib + cell, w * Fx);
                atomicAdd(sp.fib + N + cell, w * Fy);
                touch(sp, cell, stamp);
            }
        }
    }
    return m.ok && (in_tile || !t.use);
}

// Load the CTA's capsule; false (after flagging) when its parameters are out of range.
__device__ __forceinline__ bool load_ring(const Nodes& nd, const CapSmem& sm, int max_n, CapsuleParams& P,
                                          unsigned* status) {
    P = nd.caps[blockIdx.x];
    if (P.n < 3 || P.n > max_n || P.off < 0 || P.off + P.n > nd.count) {
        if (threadIdx.x == 0) atomicOr(status, kStatRing);
        return false;
    }
    for (int v = threadIdx.x; v < P.n; v += blockDim.x) sm.X[v] = nd.X[P.off + v];
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------------
// Dynamic IB (Section 2.3.2), steps 1-3: U = I(u^n) with half of the last spread
// force, F_l = u_v - U, spread with c_l = (l_left + l_right)/2. First step of a vertex:
// u_v = U and X^{-1} = X^0 - U.
// ---------------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(128) k_dyn_force_spread(const S* __restrict__ src, Lat L,
                                                          const double* __restrict__ fib_prev, Nodes nd, int max_n,
                                                          int tile_cells, Spread sp, unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    CapsuleParams P;
    if (!load_ring(nd, sm, max_n, P, status)) return;
    const int n = P.n, off = P.off;
    Tile<C> t = make_tile<C>(sm, n, 1, tile_cells, true, true);
    if (t.use) {
        fill_moments<S>(t, src, L, fib_prev);
        zero_forces<C>(t);
    }
    __syncthreads();
    // element lengths, once per element (c_l of reading R4)
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const double2 d = sm.X[v + 1 == n ? 0 : v + 1] - sm.X[v];
        sm.sst[v] = sqrt(d.x * d.x + d.y * d.y);
    }
    __syncthreads();
    const int stamp = *sp.stamp + 1;
    bool ok = true;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const double2 Xv = sm.X[v];
        // shape functions at X^n: used for U, for the spread, and by this step's update
        const MlsW<C> m = mls_setup<C>(L, Xv.x, Xv.y);
        reinterpret_cast<MlsW<C>*>(nd.mls)[off + v] = m;
        InterpT<C> o;
        ok &= interp_with<S, false>(m, t, src, L, fib_prev, o);
        const double Ux = (double)o.ux, Uy = (double)o.uy;
        double2 uv = nd.uv[off + v];
        if (nd.age[off + v] == 0) {
            uv = make_double2(Ux, Uy);
            nd.uv[off + v] = uv;
            nd.Xm1[off + v] = Xv - uv;
        }
        const double cl = 0.5 * (sm.sst[v == 0 ? n - 1 : v - 1] + sm.sst[v]);
        if (nd.Flc) nd.Flc[off + v] = make_double2(cl * (uv.x - Ux), cl * (uv.y - Uy));
        ok &= spread_with<C>(m, t, L, sp, stamp, uv.x - Ux, uv.y - Uy, cl);
    }
    __syncthreads();
    if (t.use) flush_forces<C>(t, L, sp, stamp, reinterpret_cast<int*>(sm.red));
    if (!ok) atomicOr(status, kStatSupport);
}

// Dynamic IB steps 5-8 for one capsule per CTA: xdot_0 = I(u^{n+1}) at X^n, probe
// tractions (Eq. 15-16), internal forces (Eq. 11, 13, 14), Verlet position (Eq. 23) and
// BDF2 velocity (Eq. 24).
template <typename S>
__global__ void __launch_bounds__(128) k_dyn_update(const S* __restrict__ dst, Lat L,
                                                    const double* __restrict__ fib, Nodes nd, int max_n,
                                                    int tile_cells, int* reset_count, unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    if (blockIdx.x == 0 && threadIdx.x == 0 && reset_count) *reset_count = 0;
    CapsuleParams P;
    if (!load_ring(nd, sm, max_n, P, status)) return;
    const int n = P.n, off = P.off;
    Tile<C> t = make_tile<C>(sm, n, 3, tile_cells, true, false);
    if (t.use) fill_moments<S>(t, dst, L, fib);
    __syncthreads();
    bool ok = true;
    double area2[1] = {0.0};
    const C nu = C(L.nu);
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const double2 Xv = sm.X[v], Xr = sm.X[v + 1 == n ? 0 : v + 1];
        InterpT<C> o;
        ok &= interp_with<S, false>(reinterpret_cast<const MlsW<C>*>(nd.mls)[off + v], t, dst, L, fib, o);
        sm.xd[v] = make_double2((double)o.ux, (double)o.uy);
        // element v: probes at the centroid +/- 1.2 n+ (Section 2.2.2)
        const double2 d = Xr - Xv;
        const double rl = rsqrt(d.x * d.x + d.y * d.y);
        const double npx = d.y * rl, npy = -d.x * rl;
        const double cx = 0.5 * (Xv.x + Xr.x), cy = 0.5 * (Xv.y + Xr.y);
        InterpT<C> op, om;
        ok &= interp_at<S, true>(t, dst, L, fib, cx + 1.2 * npx, cy + 1.2 * npy, op);
        ok &= interp_at<S, true>(t, dst, L, fib, cx - 1.2 * npx, cy - 1.2 * npy, om);
        // tau = rho nu (grad u + grad u^T) at each probe; Eq. 15 + Eq. 16 (per unit
        // length, then times the element length)
        const C mp = op.rho * nu, mm = om.rho * nu;
        const C txx = C(2) * (mp * op.dudx - mm * om.dudx);
        const C tyy = C(2) * (mp * op.dvdy - mm * om.dvdy);
        const C txy = mp * (op.dudy + op.dvdx) - mm * (om.dudy + om.dvdx);
        const C dp = op.p - om.p;
        const C nx = C(npx), ny = C(npy);
        const double len = (d.x * d.x + d.y * d.y) * rl;
        sm.ext[v] = make_double2((double)(-dp * nx + txx * nx + txy * ny) * len,
                                 (double)(-dp * ny + txy * nx + tyy * ny) * len);
        area2[0] += ring_terms(sm, P, nd, v);
    }
    block_reduce<1, false>(area2, sm.red);
    const double A = 0.5 * area2[0];
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const int vl = v == 0 ? n - 1 : v - 1;
        const double2 Fi = node_internal_force(sm, P, v, A);
        double2 Fe = 0.5 * (sm.ext[v] + sm.ext[vl]);
        if (nd.Fpp) Fe = Fe + nd.Fpp[off + v];   // Eq. 27, part of the total force (step 7)
        const double2 Xv = sm.X[v];
        const double2 Xm = nd.Xm1[off + v];
        const double2 xd = sm.xd[v];
        const double hm = 0.5 / P.m;
        const double2 Xn = make_double2(Xv.x + xd.x + hm * (Fi.x + Fe.x), Xv.y + xd.y + hm * (Fi.y + Fe.y));
        nd.uv[off + v] = make_double2(1.5 * Xn.x - 2.0 * Xv.x + 0.5 * Xm.x, 1.5 * Xn.y - 2.0 * Xv.y + 0.5 * Xm.y);
        nd.Xm1[off + v] = Xv;
        nd.X[off + v] = Xn;
        nd.Fint[off + v] = Fi;
        nd.Fext[off + v] = Fe;
        nd.age[off + v] += 1;
    }
    if (!ok) atomicOr(status, kStatSupport);
}

// ---------------------------------------------------------------------------------
// Kinematic IB (Section 2.4), steps i-iii: internal forces at X^n (Eq. 11, 13, 14) and
// their spread with c_v = 1.
// ---------------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(128) k_kin_force_spread(Lat L, Nodes nd, int max_n, int tile_cells, Spread sp,
                                                          unsigned* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    CapsuleParams P;
    if (!load_ring(nd, sm, max_n, P, status)) return;
    const int n = P.n, off = P.off;
    Tile<C> t = make_tile<C>(sm, n, 1, tile_cells, false, true);
    if (t.use) zero_forces<C>(t);
    double area2[1] = {0.0};
    for (int v = threadIdx.x; v < n; v += blockDim.x) area2[0] += ring_terms(sm, P, nd, v);
    block_reduce<1, false>(area2, sm.red);  // also orders the tile zeroing before the spread
    const double A = 0.5 * area2[0];
    const int stamp = *sp.stamp + 1;
    bool ok = true;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const double2 F = node_internal_force(sm, P, v, A);
        nd.Fint[off + v] = F;
        const double2 Fp = nd.Fpp ? nd.Fpp[off + v] : make_double2(0.0, 0.0);   // Eq. 27
        nd.Fext[off + v] = make_double2(0.0, 0.0);
        const MlsW<C> m = mls_setup<C>(L, sm.X[v].x, sm.X[v].y);
        reinterpret_cast<MlsW<C>*>(nd.mls)[off + v] = m;
        ok &= spread_with<C>(m, t, L, sp, stamp, F.x + Fp.x, F.y + Fp.y, 1.0);
    }
    __syncthreads();
    if (t.use) flush_forces<C>(t, L, sp, stamp, reinterpret_cast<int*>(sm.red));
    if (!ok) atomicOr(status, kStatSupport);
}

// Kinematic IB steps vii-viii: xdot = I(u^{n+1}) at X^n with half the spread force,
// X^{n+1} = 2/3 (2 X^n - X^{n-1}/2 + xdot) (Eq. 25); forward Euler on a first step.
template <typename S>
__global__ void __launch_bounds__(128) k_kin_advance(const S* __restrict__ dst, Lat L,
                                                     const double* __restrict__ fib, Nodes nd, int max_n,
                                                     int tile_cells, int* reset_count, unsigned* status) {
    using C = typename St<S>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    if (blockIdx.x == 0 && threadIdx.x == 0 && reset_count) *reset_count = 0;
    CapsuleParams P;
    if (!load_ring(nd, sm, max_n, P, status)) return;
    const int n = P.n, off = P.off;
    Tile<C> t = make_tile<C>(sm, n, 1, tile_cells, true, false);
    if (t.use) fill_moments<S>(t, dst, L, fib);
    __syncthreads();
    bool ok = true;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const double2 Xv = sm.X[v];
        InterpT<C> o;
        ok &= interp_with<S, false>(reinterpret_cast<const MlsW<C>*>(nd.mls)[off + v], t, dst, L, fib, o);
        const double Ux = (double)o.ux, Uy = (double)o.uy;
        double2 Xn;
        if (nd.age[off + v] == 0) {
            Xn = make_double2(Xv.x + Ux, Xv.y + Uy);
        } else {
            const double2 Xm = nd.Xm1[off + v];
            Xn = make_double2((2.0 / 3.0) * (2.0 * Xv.x - 0.5 * Xm.x + Ux),
                              (2.0 / 3.0) * (2.0 * Xv.y - 0.5 * Xm.y + Uy));
        }
        nd.Xm1[off + v] = Xv;
        nd.X[off + v] = Xn;
        nd.uv[off + v] = make_double2(Ux, Uy);
        nd.age[off + v] += 1;
    }
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
static size_t smem_bytes(int max_n, int cells, bool moments, bool forces) {
    return ring_smem_bytes(max_n) + tile_bytes<C>(cells, moments, forces);
}

int tile_budget(int max_n, double extent) {
    // any rotation of the reference ring, probes and supports (3 nodes each side), and
    // room for deformation
    const double side = extent + 8.0;
    long long cells = (long long)(1.5 * side * side);
    if (cells < 256) cells = 256;
    const size_t free_b = kSmemLimit - ring_smem_bytes(max_n);
    const long long cap = (long long)(free_b / (3 * sizeof(double) + 2 * sizeof(double)));
    if (cells > cap) cells = cap;
    return (int)cells;
}

void set_capsule_smem_limits(int max_n, int cells) {
#define LBMIB_SMEM(K, C, M, F) \
    cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<C>(max_n, cells, M, F))
    LBMIB_SMEM(k_dyn_force_spread<double>, double, true, true);
    LBMIB_SMEM(k_dyn_force_spread<float>, float, true, true);
    LBMIB_SMEM(k_dyn_force_spread<__half>, float, true, true);
    LBMIB_SMEM(k_dyn_update<double>, double, true, false);
    LBMIB_SMEM(k_dyn_update<float>, float, true, false);
    LBMIB_SMEM(k_dyn_update<__half>, float, true, false);
    LBMIB_SMEM(k_kin_advance<double>, double, true, false);
    LBMIB_SMEM(k_kin_advance<float>, float, true, false);
    LBMIB_SMEM(k_kin_advance<__half>, float, true, false);
    LBMIB_SMEM(k_kin_force_spread<double>, double, false, true);
    LBMIB_SMEM(k_kin_force_spread<float>, float, false, true);
#undef LBMIB_SMEM
}

template <typename S>
void launch_dyn_force_spread(const void* src, const Lat& L, const double* fib_prev, Nodes nd, int ncaps, int max_n,
                             int cells, Spread sp, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    k_dyn_force_spread<S><<<ncaps, 128, smem_bytes<C>(max_n, cells, true, true), s>>>(
        (const S*)src, L, fib_prev, nd, max_n, cells, sp, status);
}

template <typename S>
void launch_dyn_update(const void* dst, const Lat& L, const double* fib_cur, Nodes nd, int ncaps, int max_n,
                       int cells, int* reset_count, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    k_dyn_update<S><<<ncaps, 128, smem_bytes<C>(max_n, cells, true, false), s>>>(
        (const S*)dst, L, fib_cur, nd, max_n, cells, reset_count, status);
}

void launch_kin_force_spread(const Lat& L, Nodes nd, int ncaps, int max_n, int cells, Spread sp, unsigned* status,
                             bool fp64_weights, cudaStream_t s) {
    // double MLS weights when the populations are double, float otherwise
    if (fp64_weights)
        k_kin_force_spread<double><<<ncaps, 128, smem_bytes<double>(max_n, cells, false, true), s>>>(
            L, nd, max_n, cells, sp, status);
    else
        k_kin_force_spread<float><<<ncaps, 128, smem_bytes<float>(max_n, cells, false, true), s>>>(
            L, nd, max_n, cells, sp, status);
}

template <typename S>
void launch_kin_advance(const void* dst, const Lat& L, const double* fib_cur, Nodes nd, int ncaps, int max_n,
                        int cells, int* reset_count, unsigned* status, cudaStream_t s) {
    using C = typename St<S>::C;
    k_kin_advance<S><<<ncaps, 128, smem_bytes<C>(max_n, cells, true, false), s>>>(
        (const S*)dst, L, fib_cur, nd, max_n, cells, reset_count, status);
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
    template void launch_dyn_force_spread<S>(const void*, const Lat&, const double*, Nodes, int, int, int,   \
                                             Spread, unsigned*, cudaStream_t);                               \
    template void launch_dyn_update<S>(const void*, const Lat&, const double*, Nodes, int, int, int, int*,   \
                                       unsigned*, cudaStream_t);                                             \
    template void launch_kin_advance<S>(const void*, const Lat&, const double*, Nodes, int, int, int, int*,  \
                                        unsigned*, cudaStream_t);                                            \
    template void launch_interp_points<S>(const void*, const Lat&, const double*, const double2*, int,       \
                                          double*, unsigned*, cudaStream_t);

LBMIB_INSTANTIATE_IB(double)
LBMIB_INSTANTIATE_IB(float)
LBMIB_INSTANTIATE_IB(__half)

}  // namespace lbmib
