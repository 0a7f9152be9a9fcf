// Adjoint (reverse-mode derivative) of the coupled step: gradients of a capsule objective
// J(X^T) (Taylor deformation D or centroid coordinate, Section 3.1) with respect to the
// membrane constants k_s, k_b of every capsule and the uniform body force g, over T
// steps from the current state, for the Kinematic scheme (Section 2.4, steps i-viii;
// Eq. 1-14, 25; below) and the Dynamic scheme (Section 2.3.2; further down).
//
// Kinematic forward step n (populations stored post-collision, s^n = pull(post^n) the streamed
// populations that step n collides):
//   F_v   = F(X^n; k_s, k_b, k_a)                      membrane force (Eq. 11, 13, 14)
//   fib   = sum_v phi(X^n_v) F_v                       spread (step iii)
//   post^{n+1} = Coll(s^n, g + fib)                    BGK + Guo (Eq. 2, 4, 5)
//   U_v   = sum_k phi_k(X^n_v) u_k(s^{n+1}, g + fib)   interpolation (Eq. 8, Eq. 7 velocity)
//   X^{n+1} = 2/3 (2 X^n - X^{n-1}/2 + U)              Eq. 25 (forward Euler on a first step)
// Reverse step n, carrying S = dJ/ds^{n+1}, Xc = dJ/dX^{n+1}, Xp = dJ/dX^n (via X^{n-1}):
//   R0  recompute F_v and fib at X^n
//   R1  advance and interpolation transposes: U-bar, X-bar, S += du/ds, fib-bar
//   R2  lattice transpose: gather S over the streaming, node-local collision transpose,
//       F-bar = d/dF at every node, g-bar += sum F-bar
//   R3  spread transpose and membrane transpose. F = -grad E for an energy E (stretch,
//       bending and area terms are each a gradient), so dF/dX is symmetric and its
//       transpose applied to F-bar is the directional derivative of F along F-bar,
//       evaluated exactly with dual numbers.
// The derivative ignores the jumps of the MLS support when a vertex crosses a half-
// integer line (the shape functions are differentiated on the support in use).
//
// Memory: the caller's workspace holds checkpoints every K steps and a tape of K + 1
// population buffers and vertex positions; each segment is recomputed from its
// checkpoint into the tape before its reverse sweep. With K >= T the forward writes the
// tape directly and nothing is recomputed.
#include <cmath>
#include <map>
#include <cstring>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "ctx.cuh"
#include "ring.cuh"

namespace lbmib {
namespace {

// ---------------------------------------------------------------------------------
// Dual numbers: a value and its derivative along one direction.
// ---------------------------------------------------------------------------------
struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual mk(double v, double d = 0.0) { return Dual{v, d}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator+(Dual a, double s) { return {a.v + s, a.d}; }
__device__ __forceinline__ Dual operator-(double s, Dual a) { return {s - a.v, -a.d}; }
__device__ __forceinline__ Dual dsqrt(Dual a) {
    const double r = sqrt(a.v);
    return {r, a.d / (2.0 * r)};
}
__device__ __forceinline__ Dual dexp(Dual a) {
    const double e = exp(a.v);
    return {e, e * a.d};
}
__device__ __forceinline__ double vpart(Dual a) { return a.v; }
__device__ __forceinline__ double vpart(double a) { return a; }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double dexp(double a) { return exp(a); }

// A value with its derivatives along K directions at once (one pass instead of K when
// the value parts, exponentials included, would be the same in each), in the real type
// R (float for single-precision storage, double otherwise).
template <typename R, int K>
struct DN {
    R v, d[K];
};
template <typename R>
using D4 = DN<R, 4>;
template <typename R>
__device__ __forceinline__ D4<R> d4(R v) { return D4<R>{v, {R(0), R(0), R(0), R(0)}}; }
template <typename R, int K>
__device__ __forceinline__ DN<R, K> operator+(DN<R, K> a, DN<R, K> b) {
    DN<R, K> r{a.v + b.v, {}};
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <typename R, int K>
__device__ __forceinline__ DN<R, K> operator-(DN<R, K> a, DN<R, K> b) {
    DN<R, K> r{a.v - b.v, {}};
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <typename R, int K>
__device__ __forceinline__ DN<R, K> operator-(DN<R, K> a) {
    DN<R, K> r{-a.v, {}};
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = -a.d[k];
    return r;
}
template <typename R, int K>
__device__ __forceinline__ DN<R, K> operator*(DN<R, K> a, DN<R, K> b) {
    DN<R, K> r{a.v * b.v, {}};
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <typename R, int K>
__device__ __forceinline__ DN<R, K> operator/(DN<R, K> a, DN<R, K> b) {
    const R q = a.v / b.v, ib = R(1) / b.v;
    DN<R, K> r{q, {}};
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = (a.d[k] - q * b.d[k]) * ib;
    return r;
}
template <typename R, int K>
__device__ __forceinline__ DN<R, K> operator*(R s, DN<R, K> a) {
    DN<R, K> r{s * a.v, {}};
#pragma unroll
    for (int k = 0; k < K; k++) r.d[k] = s * a.d[k];
    return r;
}
template <typename R, int K>
__device__ __forceinline__ DN<R, K> operator+(DN<R, K> a, R s) { a.v += s; return a; }
template <typename R, int K>
__device__ __forceinline__ DN<R, K> dsqrt(DN<R, K> a) {
    const R r = sqrt(a.v), h = R(0.5) / r;
    DN<R, K> o{r, {}};
#pragma unroll
    for (int k = 0; k < K; k++) o.d[k] = a.d[k] * h;
    return o;
}
template <typename R, int K>
__device__ __forceinline__ DN<R, K> dexp(DN<R, K> a) {
    const R e = exp(a.v);
    DN<R, K> o{e, {}};
#pragma unroll
    for (int k = 0; k < K; k++) o.d[k] = e * a.d[k];
    return o;
}
__device__ __forceinline__ float dexp(float a) { return expf(a); }

// Real type underlying a scalar type (for constants in templated arithmetic).
template <typename T> struct RealOf { using type = T; };
template <typename R, int K> struct RealOf<DN<R, K>> { using type = R; };
template <> struct RealOf<Dual> { using type = double; };

template <typename T>
struct P2 {
    T x, y;
};
template <typename T>
__device__ __forceinline__ P2<T> operator-(P2<T> a, P2<T> b) { return {a.x - b.x, a.y - b.y}; }

// ---------------------------------------------------------------------------------
// MLS shape functions (Eq. 8-9) with their derivatives in the marker position. Along
// one axis, with offsets d_a = c + a - 1 - X of the support nodes and weights w_a =
// exp(-d_a^2 / (r_w alpha)^2):
//   q_a = w_a / S0                    (S0 = sum w, normalised weights)
//   h_a = q_a - m w_a (d_a - m) / V   (m = sum w d / S0, V = sum w (d - m)^2)
//   g_a = w_a (d_a - m) / V           (slope of the linear fit)
// and the 2-D linear-basis shape function is phi_ab = h^x_a q^y_b + q^x_a h^y_b -
// q^x_a q^y_b, the fitted x-slope weight g^x_a q^y_b and the y-slope weight q^x_a g^y_b
// (the closed-form MLS solve of the forward kernels written per axis).
// Evaluated on duals with d(d_a)/dX = -1 they give d(phi)/dX and d(phi)/dY.
// ---------------------------------------------------------------------------------
template <typename T>
struct Axis {
    T q[3], h[3], g[3];   // normalised weights, linear-fit value weights, slope weights
};

template <typename T>
__device__ Axis<T> mls_axis(T d0) {
    using R = typename RealOf<T>::type;
    T w[3], d[3];
    T s0 = T{R(0)}, s1 = T{R(0)};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        d[a] = d0 + R(a - 1);
        w[a] = dexp(R(-kMlsInvLen2) * (d[a] * d[a]));
        s0 = s0 + w[a];
        s1 = s1 + w[a] * d[a];
    }
    const T m = s1 / s0;
    T V = T{R(0)};
#pragma unroll
    for (int a = 0; a < 3; a++) V = V + w[a] * ((d[a] - m) * (d[a] - m));
    Axis<T> r;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        r.q[a] = w[a] / s0;
        r.h[a] = r.q[a] - (m * w[a] * (d[a] - m)) / V;
        r.g[a] = (w[a] * (d[a] - m)) / V;
    }
    return r;
}

// Threads per CTA of the interpolation transposes (one thread per vertex and support
// node, mapped over the whole grid): small CTAs spread a few capsules over many SMs.
constexpr int kInterpThreads = 64;

struct Shape {
    int cx, cy;
    bool ok;
    double phi[3][3], px[3][3], py[3][3];   // [b][a]: value, d/dX, d/dY
};

__device__ Shape shape_with_derivatives(const Lat& L, double X, double Y) {
    Shape s;
    s.ok = support_centre(L, X, Y, s.cx, s.cy);
    const Axis<Dual> ax = mls_axis<Dual>(mk((double)s.cx - X, -1.0));
    const Axis<Dual> ay = mls_axis<Dual>(mk((double)s.cy - Y, -1.0));
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const Dual hx = ax.h[a], qx = ax.q[a], hy = ay.h[b], qy = ay.q[b];
            s.phi[b][a] = hx.v * qy.v + qx.v * hy.v - qx.v * qy.v;
            s.px[b][a] = hx.d * qy.v + qx.d * hy.v - qx.d * qy.v;
            s.py[b][a] = hx.v * qy.d + qx.v * hy.d - qx.v * qy.d;
        }
    return s;
}

__device__ __forceinline__ int support_cell(const Lat& L, const Shape& s, int a, int b) {
    return support_row(L, s.cy + b - 1) * L.nx + wrapi(s.cx + a - 1, L.nx);
}

// ---------------------------------------------------------------------------------
// Membrane force of vertex v with unit constants, split into its stretch (Eq. 11),
// bending (Eq. 13) and area (Eq. 14) parts: F_v = k_s Fs + k_b Fb + k_a Fa. Written
// for any scalar type so that dual numbers give its directional derivative.
// ---------------------------------------------------------------------------------
template <typename T, typename GetX>
__device__ void membrane_parts(int v, int n, GetX X, const double* L0, const double* c0, const double* s0, T A,
                               double A0, P2<T>& Fs, P2<T>& Fb, P2<T>& Fa) {
    auto idx = [n](int k) { return k < 0 ? k + n : (k >= n ? k - n : k); };
    P2<T> p[5];   // X_{v-2} .. X_{v+2}
#pragma unroll
    for (int j = 0; j < 5; j++) p[j] = X(idx(v + j - 2));
    // stretch: elements v-1 (p1 -> p2) and v (p2 -> p3)
    {
        const P2<T> bl = p[2] - p[1], br = p[3] - p[2];
        const T ll = dsqrt(bl.x * bl.x + bl.y * bl.y), lr = dsqrt(br.x * br.x + br.y * br.y);
        const T tl = -((ll + (-L0[idx(v - 1)])) / ll), tr = -((lr + (-L0[v])) / lr);
        Fs.x = tr * (p[2].x - p[3].x) + tl * (p[2].x - p[1].x);
        Fs.y = tr * (p[2].y - p[3].y) + tl * (p[2].y - p[1].y);
    }
    // bending: angles at v-1, v, v+1 (centres p[1], p[2], p[3])
    T bs[3];
    P2<T> bdl[3], bdr[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const P2<T> a = p[j + 1] - p[j], b = p[j + 2] - p[j + 1];
        const T a2 = a.x * a.x + a.y * a.y, b2 = b.x * b.x + b.y * b.y;
        const T cr = a.x * b.y - a.y * b.x, dt = a.x * b.x + a.y * b.y;
        const int k = idx(v + j - 1);
        bs[j] = (c0[k] * cr - s0[k] * dt) / dsqrt(a2 * b2);
        bdl[j] = {(-a.y) / a2, a.x / a2};
        bdr[j] = {(-b.y) / b2, b.x / b2};
    }
    Fb.x = bs[1] * (bdl[1].x + bdr[1].x) - bs[2] * bdl[2].x - bs[0] * bdr[0].x;
    Fb.y = bs[1] * (bdl[1].y + bdr[1].y) - bs[2] * bdl[2].y - bs[0] * bdr[0].y;
    // area: (1 - A / A0) / 6 * (dr.y + dl.y, -(dr.x + dl.x)), dr + dl = X_{v+1} - X_{v-1}
    const T fa = (1.0 / 6.0) * (1.0 - A / mk(A0));
    Fa.x = fa * (p[3].y - p[1].y);
    Fa.y = -(fa * (p[3].x - p[1].x));
}

// ---------------------------------------------------------------------------------
// Objectives (Section 3.1) of one ring, for any scalar type: Taylor deformation D from
// the area second moments, or a centroid coordinate.
// ---------------------------------------------------------------------------------
enum { kObjTaylorD = 0, kObjCentroidY = 1, kObjCentroidX = 2 };

// Contribution of the ring term (a, b) = (X_i - c, X_{i+1} - c) to the six area sums
// s = {2A, 6A xc, 6A yc, 12 Sxx, 12 Syy, 24 Sxy} (Green's theorem about a fixed point c).
template <typename T>
__device__ __forceinline__ void ring_term_sums(P2<T> a, P2<T> b, T (&s)[6]) {
    const T c = a.x * b.y - b.x * a.y;
    s[0] = s[0] + c;
    s[1] = s[1] + (a.x + b.x) * c;
    s[2] = s[2] + (a.y + b.y) * c;
    s[3] = s[3] + (a.x * a.x + a.x * b.x + b.x * b.x) * c;
    s[4] = s[4] + (a.y * a.y + a.y * b.y + b.y * b.y) * c;
    s[5] = s[5] + (a.x * b.y + 2.0 * (a.x * a.y) + 2.0 * (b.x * b.y) + b.x * a.y) * c;
}

// The objective from the six sums: centroid (offset by c) or the Taylor deformation
// from the eigenvalues of the area second-moment tensor about the centroid.
template <typename T>
__device__ T objective_from_sums(const T (&s)[6], double2 c, int kind) {
    const T A = 0.5 * s[0];
    const T cx = s[1] / (6.0 * A), cy = s[2] / (6.0 * A);
    if (kind == kObjCentroidY) return cy + c.y;
    if (kind == kObjCentroidX) return cx + c.x;
    const T Ixx = (1.0 / 12.0) * s[3] - A * (cx * cx);
    const T Iyy = (1.0 / 12.0) * s[4] - A * (cy * cy);
    const T Ixy = (1.0 / 24.0) * s[5] - A * (cx * cy);
    const T mid = 0.5 * (Ixx + Iyy);
    const T dd = dsqrt(0.25 * ((Ixx - Iyy) * (Ixx - Iyy)) + Ixy * Ixy);
    const T lmax = (mid + dd) / A, lmin = (mid - dd) / A;
    const T a = 2.0 * dsqrt(lmax);
    const T b = vpart(lmin) > 0.0 ? 2.0 * dsqrt(lmin) : T{0.0};
    return (a - b) / (a + b);
}

// J and dJ/dX of capsule `cap`. The objectives are invariant under a shift of the ring
// (the centroid shifts with it), so the sums are taken about the fixed point c = X_0 and
// dJ/dX_v = sum_k dJ/ds_k ds_k/dX_v, where only the two ring terms that hold X_v
// depend on it: O(n) work. One block.
__global__ void k_adj_objective(Nodes nd, int cap, int kind, double2* xc, double* J) {
    __shared__ double red[32 * 8];
    const CapsuleParams P = nd.caps[cap];
    const int n = P.n;
    const double2* X = nd.X + P.off;
    const double2 c = X[0];
    auto rel = [&](int i) { return P2<double>{X[i].x - c.x, X[i].y - c.y}; };
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) ring_term_sums<double>(rel(i), rel(i + 1 == n ? 0 : i + 1), s);
    block_reduce<6, false>(s, red);
    if (threadIdx.x == 0) *J = objective_from_sums<double>(s, c, kind);
    double dJ[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        Dual sd[6];
#pragma unroll
        for (int m = 0; m < 6; m++) sd[m] = mk(s[m], m == k ? 1.0 : 0.0);
        dJ[k] = objective_from_sums<Dual>(sd, c, kind).d;
    }
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const P2<double> xl = rel(v == 0 ? n - 1 : v - 1), xv = rel(v), xr = rel(v + 1 == n ? 0 : v + 1);
        double g[2];
#pragma unroll
        for (int comp = 0; comp < 2; comp++) {
            const P2<Dual> dv{mk(xv.x, comp == 0 ? 1.0 : 0.0), mk(xv.y, comp == 1 ? 1.0 : 0.0)};
            Dual ds[6] = {mk(0.0), mk(0.0), mk(0.0), mk(0.0), mk(0.0), mk(0.0)};
            ring_term_sums<Dual>(P2<Dual>{mk(xl.x), mk(xl.y)}, dv, ds);
            ring_term_sums<Dual>(dv, P2<Dual>{mk(xr.x), mk(xr.y)}, ds);
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < 6; k++) t += dJ[k] * ds[k].d;
            g[comp] = t;
        }
        xc[P.off + v] = make_double2(g[0], g[1]);
    }
}

// ---------------------------------------------------------------------------------
// R0: membrane forces at X^n (saved per vertex) and their spread into the force field.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_adj_spread(Lat L, Nodes nd, const double2* Xn, int max_n, double2* Fv,
                                                    Shape* shp, double* fib) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    const CapsuleParams P = nd.caps[blockIdx.x];
    if (P.n < 3 || P.n > max_n) return;
    const int n = P.n, off = P.off;
    for (int v = threadIdx.x; v < n; v += blockDim.x) sm.X[v] = Xn[off + v];
    __syncthreads();
    double area2[1] = {0.0};
    for (int v = threadIdx.x; v < n; v += blockDim.x) area2[0] += ring_terms(sm, P, nd, v);
    block_reduce<1, false>(area2, sm.red);
    const long long N = (long long)L.nx * L.ny;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const double2 F = node_internal_force(sm, P, v, 0.5 * area2[0]);
        Fv[off + v] = F;
        const Shape s = shape_with_derivatives(L, sm.X[v].x, sm.X[v].y);
        shp[off + v] = s;   // reused by the interpolation and spread transposes
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int cell = support_cell(L, s, a, b);
                atomicAdd(fib + cell, s.phi[b][a] * F.x);
                atomicAdd(fib + N + cell, s.phi[b][a] * F.y);
            }
    }
}

// ---------------------------------------------------------------------------------
// R1: transposes of the advance (Eq. 25) and of the interpolation (Eq. 8 with the Eq. 7
// velocity u_k = (m_k + (g + fib_k)/2) / rho_k at the support nodes). One thread per
// (vertex, support node); X-bar of X^n accumulates in xnew (zero on entry), completed
// by R3.
// ---------------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(kInterpThreads) k_adj_interp(Lat L, const S* __restrict__ post1,
                                                    const double* __restrict__ fib, const Shape* __restrict__ shp,
                                                    const int* age0, int nloc, int count, const double2* xc,
                                                    double2* xp, double2* xnew, double* sbar,
                                                    double* bbar, double* grad_g, unsigned* status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = t / 9, k = t - 9 * (t / 9);
    double gsx = 0.0, gsy = 0.0;
    if (v < count) {
        const bool first = age0[v] + nloc == 0;
        const double2 c = xc[v];
        const double kU = first ? 1.0 : 2.0 / 3.0;
        const double Ux = kU * c.x, Uy = kU * c.y;
        if (k == 0) {
            const double kX = first ? 1.0 : 4.0 / 3.0;
            const double2 p = xp[v];
            atomicAdd(&xnew[v].x, p.x + kX * c.x);
            atomicAdd(&xnew[v].y, p.y + kX * c.y);
            xp[v] = first ? make_double2(0.0, 0.0) : make_double2(-c.x / 3.0, -c.y / 3.0);
            if (!shp[v].ok) atomicOr(status, kStatSupport);
        }
        const int a = k % 3, b = k / 3;
        const Shape& s = shp[v];
        const long long N = (long long)L.nx * L.ny;
        const int xk = wrapi(s.cx + a - 1, L.nx), yk = support_row(L, s.cy + b - 1);
        const long long cell = (long long)yk * L.nx + xk;
        typename St<S>::C qc[9];
        pull_all<S>(post1, L, xk, yk, qc);
        double q[9];
#pragma unroll
        for (int i = 0; i < 9; i++) q[i] = (double)qc[i];
        double drho = 0.0, mx = 0.0, my = 0.0;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            drho += q[i];
            mx += ex(i) * q[i];
            my += ey(i) * q[i];
        }
        const double rho = 1.0 + drho;
        const double ux = (mx + 0.5 * (L.gx + fib[cell])) / rho;
        const double uy = (my + 0.5 * (L.gy + fib[N + cell])) / rho;
        const double uU = ux * Ux + uy * Uy;
        atomicAdd(&xnew[v].x, s.px[b][a] * uU);
        atomicAdd(&xnew[v].y, s.py[b][a] * uU);
        const double cf = s.phi[b][a] / rho;
#pragma unroll
        for (int i = 0; i < 9; i++)
            atomicAdd(sbar + (long long)i * N + cell, cf * ((ex(i) - ux) * Ux + (ey(i) - uy) * Uy));
        atomicAdd(bbar + cell, 0.5 * cf * Ux);
        atomicAdd(bbar + N + cell, 0.5 * cf * Uy);
        gsx = 0.5 * cf * Ux;
        gsy = 0.5 * cf * Uy;
    }
    for (int o = 16; o > 0; o >>= 1) {
        gsx += __shfl_xor_sync(0xffffffffu, gsx, o);
        gsy += __shfl_xor_sync(0xffffffffu, gsy, o);
    }
    if ((threadIdx.x & 31) == 0 && (gsx != 0.0 || gsy != 0.0)) {
        atomicAdd(grad_g, gsx);
        atomicAdd(grad_g + 1, gsy);
    }
}

// ---------------------------------------------------------------------------------
// R2: lattice transpose of step n. Each post-collision population post_j(x) feeds
// exactly one streamed population: s_j(x + e_j), or s_opp(j)(x) where x + e_j lies
// beyond a wall, so its adjoint is a gather. The collision (BGK + Guo, Eq. 2, 4, 5) is
// node-local; its transpose is written out term by term (reverse order of the forward
// evaluation). Also clears the other parity of the force-field buffers.
// ---------------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void collide_adjoint(const C s[9], C Fx, C Fy, C omega, const C pb[9], C sb[9], C& Fbx,
                                                C& Fby) {
    C drho, mx, my;
    moments<C>(s, drho, mx, my);
    const C rho = C(1) + drho;
    const C ux = (mx + C(0.5) * Fx) / rho, uy = (my + C(0.5) * Fy) / rho;
    const C usq = ux * ux + uy * uy;
    const C cf = C(1) - C(0.5) * omega;
    C drho_b = 0, rho_b = 0, usq_b = 0, uF_b = 0, ux_b = 0, uy_b = 0;
    Fbx = 0;
    Fby = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const C w = wgt<C>(i);
        const C eu = C(ex(i)) * ux + C(ey(i)) * uy;
        const C eF = C(ex(i)) * Fx + C(ey(i)) * Fy;
        const C seq_b = omega * pb[i];
        const C Fi_b = pb[i];
        sb[i] = (C(1) - omega) * pb[i];
        drho_b += w * seq_b;
        rho_b += w * seq_b * (eu * (C(3) + C(4.5) * eu) - C(1.5) * usq);
        usq_b -= C(1.5) * rho * w * seq_b;
        const C eu_b = w * seq_b * rho * (C(3) + C(9) * eu) + C(9) * cf * w * Fi_b * eF;
        const C eF_b = cf * w * Fi_b * (C(3) + C(9) * eu);
        uF_b -= C(3) * cf * w * Fi_b;
        ux_b += C(ex(i)) * eu_b;
        uy_b += C(ey(i)) * eu_b;
        Fbx += C(ex(i)) * eF_b;
        Fby += C(ey(i)) * eF_b;
    }
    // uF = ux Fx + uy Fy; usq = ux^2 + uy^2
    ux_b += uF_b * Fx + C(2) * ux * usq_b;
    uy_b += uF_b * Fy + C(2) * uy * usq_b;
    Fbx += uF_b * ux;
    Fby += uF_b * uy;
    // u = (m + F/2) / rho
    const C mx_b = ux_b / rho, my_b = uy_b / rho;
    Fbx += C(0.5) * mx_b;
    Fby += C(0.5) * my_b;
    rho_b -= (ux_b * ux + uy_b * uy) / rho;
    drho_b += rho_b;
#pragma unroll
    for (int i = 0; i < 9; i++) sb[i] += drho_b + C(ex(i)) * mx_b + C(ey(i)) * my_b;
}

template <typename S>
__global__ void __launch_bounds__(256) k_adj_lattice(const S* __restrict__ post0, Lat L,
                                                     const double* __restrict__ sb_in, double* __restrict__ sb_out,
                                                     double* __restrict__ fbar, const double* __restrict__ fib,
                                                     double* fib_clear, double* bbar_clear, double* grad_g) {
    using C = double;   // adjoint fields are double in every storage mode
    __shared__ double red[2 * 32];
    const long long N = (long long)L.nx * L.ny;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double gx = 0.0, gy = 0.0;
    if (node < N) {
        const int y = (int)(node / L.nx), x = (int)(node - (long long)y * L.nx);
        C pb[9], s[9], sb[9];
#pragma unroll
        for (int j = 0; j < 9; j++) {
            const int ty = y + ey(j);
            if (L.walls && (ty < 0 || ty >= L.ny)) {
                pb[j] = sb_in[(long long)opp(j) * N + node];
            } else {
                const int tx = wrapi(x + ex(j), L.nx);
                pb[j] = sb_in[(long long)j * N + (long long)wrapi(ty, L.ny) * L.nx + tx];
            }
        }
        typename St<S>::C sc[9];
        pull_all<S>(post0, L, x, y, sc);
        const double Fx = L.gx + fib[node], Fy = L.gy + fib[N + node];
        C Fbx, Fby;
        if constexpr (sizeof(typename St<S>::C) == 8) {
#pragma unroll
            for (int i = 0; i < 9; i++) s[i] = (double)sc[i];
            collide_adjoint<double>(s, Fx, Fy, L.omega, pb, sb, Fbx, Fby);
        } else {
            // The collision keeps mass (sum of the outgoing populations = sum of the
            // incoming ones) and momentum up to the force (sum e post = sum e s + F), so
            // the adjoint modes 1, e_x, e_y pass through it exactly: 1 -> 1 with no force
            // adjoint, e_x -> e_x with force adjoint (1, 0). Those parts are split off in
            // double (weighted mean and first moments of p-bar) and only the remainder
            // goes through the float transpose.
            double c0 = 0.0, ca = 0.0, cb = 0.0;
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const double w = wgt<double>(i);
                c0 += w * pb[i];
                ca += 3.0 * w * ex(i) * pb[i];
                cb += 3.0 * w * ey(i) * pb[i];
            }
            float sf[9], rf[9], sbf[9], fx, fy;
#pragma unroll
            for (int i = 0; i < 9; i++) {
                sf[i] = (float)sc[i];
                rf[i] = (float)(pb[i] - c0 - ca * ex(i) - cb * ey(i));
            }
            collide_adjoint<float>(sf, (float)Fx, (float)Fy, L.omegaf, rf, sbf, fx, fy);
#pragma unroll
            for (int i = 0; i < 9; i++) sb[i] = c0 + ca * ex(i) + cb * ey(i) + (double)sbf[i];
            Fbx = ca + (double)fx;
            Fby = cb + (double)fy;
        }
#pragma unroll
        for (int i = 0; i < 9; i++) sb_out[(long long)i * N + node] = sb[i];
        fbar[node] = Fbx;
        fbar[N + node] = Fby;
        fib_clear[node] = 0.0;
        fib_clear[N + node] = 0.0;
        if (bbar_clear) {   // the Dynamic sweep has no half-force adjoint
            bbar_clear[node] = 0.0;
            bbar_clear[N + node] = 0.0;
        }
        gx = (double)Fbx;
        gy = (double)Fby;
    }
    for (int o = 16; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[2 * warp] = gx;
        red[2 * warp + 1] = gy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tx = 0.0, ty = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            tx += red[2 * w];
            ty += red[2 * w + 1];
        }
        atomicAdd(grad_g, tx);
        atomicAdd(grad_g + 1, ty);
    }
}

// Membrane transpose of one capsule (collective): with the vertices in sm.X and F-bar in
// sm.ext, adds d/de F_v(X + e F-bar) (= (dF/dX)^T F-bar, the Jacobian being symmetric)
// to sm.xd[v], and F-bar . dF/dk to the k_s and k_b gradients of capsule `cap`.
__device__ void membrane_transpose(const CapSmem& sm, const CapsuleParams& P, const Nodes& nd, int cap, int ncaps,
                                   double* grad) {
    const int n = P.n, off = P.off;
    double ar[2] = {0.0, 0.0};
    auto getd = [&](int k) {
        const double2 p = sm.X[k], t = sm.ext[k];
        return P2<Dual>{mk(p.x, t.x), mk(p.y, t.y)};
    };
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const P2<Dual> p0 = getd(0), a = getd(v) - p0, b = getd(v + 1 == n ? 0 : v + 1) - p0;
        const Dual c2 = a.x * b.y - b.x * a.y;
        ar[0] += c2.v;
        ar[1] += c2.d;
    }
    block_reduce<2, false>(ar, sm.red);
    const Dual A = mk(0.5 * ar[0], 0.5 * ar[1]);
    double kk[2] = {0.0, 0.0};
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        P2<Dual> Fs, Fb, Fa;
        membrane_parts<Dual>(v, n, getd, nd.L0 + off, nd.c0 + off, nd.s0 + off, A, P.A0, Fs, Fb, Fa);
        const double2 fb = sm.ext[v];
        kk[0] += fb.x * Fs.x.v + fb.y * Fs.y.v;
        kk[1] += fb.x * Fb.x.v + fb.y * Fb.y.v;
        const double2 c = sm.xd[v];
        sm.xd[v] = make_double2(c.x + P.ks * Fs.x.d + P.kb * Fb.x.d + P.ka * Fa.x.d,
                                c.y + P.ks * Fs.y.d + P.kb * Fb.y.d + P.ka * Fa.y.d);
    }
    block_reduce<2, false>(kk, sm.red);
    if (threadIdx.x == 0) {
        grad[cap] += kk[0];
        grad[ncaps + cap] += kk[1];
    }
}

// ---------------------------------------------------------------------------------
// R3: spread and membrane transposes, one CTA per capsule.
//   F-bar_v = sum_k phi_k(X_v) fib-bar_k,  X-bar_v += sum_k grad phi_k (fib-bar_k . F_v)
//   X-bar_v += d/de F_v(X + e F-bar),      k_s-bar += F-bar . Fs,  k_b-bar += F-bar . Fb
// with fib-bar = (collision force adjoint) + (interpolation half-force adjoint).
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_adj_membrane(Lat L, Nodes nd, const double2* Xn, int max_n,
                                                      const double2* Fv, const Shape* __restrict__ shp,
                                                      const double* __restrict__ fbar, const double* __restrict__ bbar,
                                                      double2* xnew, double2* xc, int ncaps, double* grad) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    const int cap = blockIdx.x;
    const CapsuleParams P = nd.caps[cap];
    if (P.n < 3 || P.n > max_n) return;
    const int n = P.n, off = P.off;
    const long long N = (long long)L.nx * L.ny;
    for (int v = threadIdx.x; v < n; v += blockDim.x) sm.X[v] = Xn[off + v];
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const Shape& s = shp[off + v];
        const double2 F = Fv[off + v];
        double fbx = 0.0, fby = 0.0, gxv = 0.0, gyv = 0.0;
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int cell = support_cell(L, s, a, b);
                const double tx = fbar[cell] + bbar[cell];
                const double ty = fbar[N + cell] + bbar[N + cell];
                fbx += s.phi[b][a] * tx;
                fby += s.phi[b][a] * ty;
                const double tF = tx * F.x + ty * F.y;
                gxv += s.px[b][a] * tF;
                gyv += s.py[b][a] * tF;
            }
        sm.ext[v] = make_double2(fbx, fby);   // F-bar of vertex v
        const double2 c = xnew[off + v];
        sm.xd[v] = make_double2(c.x + gxv, c.y + gyv);
        xnew[off + v] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    membrane_transpose(sm, P, nd, cap, ncaps, grad);
    for (int v = threadIdx.x; v < n; v += blockDim.x) xc[off + v] = sm.xd[v];
}

// =================================================================================
// Dynamic scheme (Section 2.3.2, steps 1-8; Eq. 15-16, 21-24). Forward step n, every
// interpolation on the populations before any IB force (velocity (m + g/2)/rho):
//   U = I(s^n, X^n)                     (first step of a vertex: u_v := U, X^{n-1} := X^n - U)
//   F_l = u_v - U,  c_l = (l_left + l_right)/2,  fib^n = sum phi(X^n) c_l F_l
//   post^{n+1} = Coll(s^n, g + fib^n)
//   F^ext = tractions(s^{n+1}, X^n),  F^int = F(X^n)
//   X^{n+1} = X^n + U + (F^int + F^ext) / (2 m)       (Eq. 23, tentative velocity U)
//   u_v^{n+1} = 3/2 X^{n+1} - 2 X^n + 1/2 X^{n-1}                             (Eq. 24)
// The reverse sweep carries S = dJ/ds^{n+1}, Xc = dJ/dX^{n+1}, Xm = dJ/dX^n through the
// X^{n-1} slot and Ub = dJ/du_v^{n+1}.
// =================================================================================

// MLS density and velocity gradient at probe P from the fields of its 3x3 support
// (centre fixed), for any scalar type.
template <typename T>
struct ProbeVal {
    T rho, G[2][2];   // G[a][b] = d u_a / d x_b
};

template <typename T, typename F>
__device__ ProbeVal<T> probe_eval(T d0x, T d0y, const F* drho, const F* ux, const F* uy) {
    using R = typename RealOf<T>::type;
    const Axis<T> ax = mls_axis<T>(d0x), ay = mls_axis<T>(d0y);
    ProbeVal<T> o;
    o.rho = T{R(1)};
    o.G[0][0] = o.G[0][1] = o.G[1][0] = o.G[1][1] = T{R(0)};
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int k = 3 * b + a;
            const T phi = ax.h[a] * ay.q[b] + ax.q[a] * ay.h[b] - ax.q[a] * ay.q[b];
            const T gx = ax.g[a] * ay.q[b], gy = ax.q[a] * ay.g[b];
            o.rho = o.rho + R(drho[k]) * phi;
            o.G[0][0] = o.G[0][0] + R(ux[k]) * gx;
            o.G[0][1] = o.G[0][1] + R(ux[k]) * gy;
            o.G[1][0] = o.G[1][0] + R(uy[k]) * gx;
            o.G[1][1] = o.G[1][1] + R(uy[k]) * gy;
        }
    return o;
}

// Part of the traction of one element (Eq. 15-16) that comes from probe s (0: outer,
// at the centroid + 1.2 n; 1: inner, at - 1.2 n), with n = (dy, -dx)/l the outward normal
// of a counter-clockwise ring, p = rho/3 and tau = rho nu (G + G^T):
//   F = l (-(p+ - p-) n + (tau+ - tau-) n) = T_0 - T_1,  T_s = l (-p_s n + tau_s n).
// Returns (+/-) T_s for fields sampled at the probe's support; the end points are given
// relative to the support's centre node (so single precision keeps their digits). Any
// scalar type.
template <typename T, typename F>
__device__ P2<T> probe_traction(P2<T> X1, P2<T> X2, int s, const F* drho, const F* ux, const F* uy,
                                typename RealOf<T>::type nu) {
    using R = typename RealOf<T>::type;
    const P2<T> d = X2 - X1;
    const T len = dsqrt(d.x * d.x + d.y * d.y);
    const P2<T> nn{d.y / len, -(d.x / len)};
    const R sg = s == 0 ? R(1.2) : R(-1.2);
    // support offsets from the probe: centre - P = -(C + sg n) in these coordinates
    const ProbeVal<T> o = probe_eval<T, F>(-(R(0.5) * (X1.x + X2.x) + sg * nn.x),
                                           -(R(0.5) * (X1.y + X2.y) + sg * nn.y), drho, ux, uy);
    const T p = R(1.0 / 3.0) * o.rho;
    const T n_[2] = {nn.x, nn.y};
    T Fo[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        T t = -(p * n_[a]);
#pragma unroll
        for (int b = 0; b < 2; b++) t = t + nu * (o.rho * (o.G[a][b] + o.G[b][a])) * n_[b];
        Fo[a] = (s == 0 ? R(1) : R(-1)) * (len * t);
    }
    return P2<T>{Fo[0], Fo[1]};
}

// DR0: the spread force of step n-1 (and of step n at the first reverse step of a
// segment) from the taped c_l F_l, and the MLS shapes. Shapes at X^n were computed by
// the previous reverse step (as its X^{n-1}) except at a segment's first reverse step
// (compute_n); shapes at X^{n-1} are computed here for this step's spread of fib^{n-1}
// and kept for the next reverse step.
__global__ void __launch_bounds__(128) k_adjd_spread(Lat L, Nodes nd, int max_n, const double2* Xn,
                                                     const double2* Xp, const double2* Flc_n,
                                                     const double2* Flc_p, double* fib_n, double* fib_p,
                                                     Shape* shp_n, Shape* shp_p, bool compute_n) {
    const CapsuleParams P = nd.caps[blockIdx.x];
    if (P.n < 3 || P.n > max_n) return;
    const long long N = (long long)L.nx * L.ny;
    for (int v = threadIdx.x; v < P.n; v += blockDim.x) {
        const int g = P.off + v;
        if (compute_n) {
            const Shape s = shape_with_derivatives(L, Xn[g].x, Xn[g].y);
            shp_n[g] = s;
            if (fib_n) {
                const double2 F = Flc_n[g];
#pragma unroll
                for (int b = 0; b < 3; b++)
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        const int cell = support_cell(L, s, a, b);
                        atomicAdd(fib_n + cell, s.phi[b][a] * F.x);
                        atomicAdd(fib_n + N + cell, s.phi[b][a] * F.y);
                    }
            }
        }
        if (fib_p) {
            const Shape sp = shape_with_derivatives(L, Xp[g].x, Xp[g].y);
            shp_p[g] = sp;
            const double2 F = Flc_p[g];
#pragma unroll
            for (int b = 0; b < 3; b++)
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const int cell = support_cell(L, sp, a, b);
                    atomicAdd(fib_p + cell, sp.phi[b][a] * F.x);
                    atomicAdd(fib_p + N + cell, sp.phi[b][a] * F.y);
                }
        }
    }
}

// Fields (density deviation, velocity before any IB force, density) at lattice node (xk, yk).
template <typename S>
__device__ __forceinline__ void node_fields(const S* __restrict__ post, const Lat& L, int xk, int yk, double& drho,
                                            double& ux, double& uy) {
    double mx = 0.0, my = 0.0;
    drho = 0.0;
    typename St<S>::C qc[9];
    pull_all<S>(post, L, xk, yk, qc);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const double q = (double)qc[i];
        drho += q;
        mx += ex(i) * q;
        my += ey(i) * q;
    }
    const double rho = 1.0 + drho;
    ux = (mx + 0.5 * L.gx) / rho;
    uy = (my + 0.5 * L.gy) / rho;
}

// Adjoint of the fields at support node `cell`: drho-bar and u-bar into the population
// adjoint (drho = sum s, u = (m + g/2) / rho) and the body-force gradient.
__device__ __forceinline__ void inject_fields(const Lat& L, long long cell, double drho_b, double ubx, double uby,
                                              double ux, double uy, double rho, double* sbar, double& gsx,
                                              double& gsy) {
    const long long N = (long long)L.nx * L.ny;
#pragma unroll
    for (int i = 0; i < 9; i++)
        atomicAdd(sbar + (long long)i * N + cell, drho_b + ((ex(i) - ux) * ubx + (ey(i) - uy) * uby) / rho);
    gsx += 0.5 * ubx / rho;
    gsy += 0.5 * uby / rho;
}

// DR1: transposes of Eq. 24, Eq. 23 and the membrane force, one CTA per capsule. Writes
// dJ/dX^n (partial) to xout, the adjoint of Eq. 23's tentative velocity U to u2b, F^tot-bar
// to ftb (for the tractions), and keeps dJ/dX^{n-1} (from Eq. 24) in xm for DR3.
__global__ void __launch_bounds__(128) k_adjd_update(Nodes nd, int max_n, const double2* Xn, const double2* xc,
                                                     double2* xm, const double2* ub, double2* xout, double2* u2b,
                                                     double2* ftb, int ncaps, double* grad) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    const int cap = blockIdx.x;
    const CapsuleParams P = nd.caps[cap];
    if (P.n < 3 || P.n > max_n) return;
    const int n = P.n, off = P.off;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const int g = off + v;
        sm.X[v] = Xn[g];
        const double2 u = ub[g], c = xc[g];
        const double2 ct = make_double2(c.x + 1.5 * u.x, c.y + 1.5 * u.y);   // dJ/dX^{n+1} in total
        u2b[g] = ct;
        const double2 fb = make_double2(ct.x / (2.0 * P.m), ct.y / (2.0 * P.m));   // F^tot-bar
        sm.ext[v] = fb;
        ftb[g] = fb;
        const double2 m = xm[g];
        sm.xd[v] = make_double2(m.x - 2.0 * u.x + ct.x, m.y - 2.0 * u.y + ct.y);
        xm[g] = make_double2(0.5 * u.x, 0.5 * u.y);                             // dJ/dX^{n-1}
    }
    __syncthreads();
    membrane_transpose(sm, P, nd, cap, ncaps, grad);
    for (int v = threadIdx.x; v < n; v += blockDim.x) xout[off + v] = sm.xd[v];
}

// DR1t: transpose of the tractions (Eq. 15-16), nine threads per (element, probe), one
// per node of the probe's support, kTractGroups (element, probe) groups per CTA. Each end vertex
// receives half of the element force, so F_l-bar = (F^tot-bar_1 + F^tot-bar_2)/2. The
// fields enter linearly: density through p and tau, the velocity gradient through tau;
// the positions through the probe location, normal and length. Thread k of a group loads
// the fields of support node k; threads 0-3 each take the derivative along one end
// coordinate (single-lane duals, in parallel); every thread injects its own node's share
// of the field adjoints.
// (element, probe) groups per CTA, and the CTA rounded up to whole warps (the spare
// threads only join the final warp reduction): few groups per CTA spread the work over
// many SMs
constexpr int kTractGroups = 10;
constexpr int kTractThreads = (9 * kTractGroups + 31) / 32 * 32;

template <typename S>
__global__ void __launch_bounds__(kTractThreads) k_adjd_tract(Lat L, Nodes nd, int count, const double2* Xn,
                                                                 const S* __restrict__ post1, const double2* ftb,
                                                                 double2* xout, double* sbar, double* grad_g,
                                                                 unsigned* status) {
    // the traction adjoint computes in single precision for single-precision storage
    using R = typename std::conditional<sizeof(S) == 8, double, float>::type;
    __shared__ R fld[3][kTractGroups][9];   // density deviation, u_x, u_y of each support node
    const int grp = threadIdx.x / 9, k = threadIdx.x - 9 * grp;
    const int t = blockIdx.x * kTractGroups + grp;
    const int g1 = t >> 1, s = t & 1;
    const bool act = grp < kTractGroups && g1 < count;
    double gsx = 0.0, gsy = 0.0;
    bool ok = true;
    int g2 = 0, cx = 0, cy = 0;
    double2 X1{}, X2{};
    double dx = 0.0, dy = 0.0, len = 1.0, Px = 0.0, Py = 0.0, dr = 0.0, u = 0.0, w = 0.0;
    long long cell = 0;
    R Fb[2] = {R(0), R(0)};
    if (act) {
        const CapsuleParams P = nd.caps[nd.capid[g1]];
        const int v = g1 - P.off;
        g2 = P.off + (v + 1 == P.n ? 0 : v + 1);
        X1 = Xn[g1];
        X2 = Xn[g2];
        const double2 f1 = ftb[g1], f2 = ftb[g2];
        Fb[0] = R(0.5 * (f1.x + f2.x));
        Fb[1] = R(0.5 * (f1.y + f2.y));
        dx = X2.x - X1.x;
        dy = X2.y - X1.y;
        len = sqrt(dx * dx + dy * dy);
        const double sg = s == 0 ? 1.2 : -1.2;
        Px = 0.5 * (X1.x + X2.x) + sg * dy / len;
        Py = 0.5 * (X1.y + X2.y) - sg * dx / len;
        ok = support_centre(L, Px, Py, cx, cy);
        const int xk = wrapi(cx + k % 3 - 1, L.nx), yk = support_row(L, cy + k / 3 - 1);
        cell = (long long)yk * L.nx + xk;
        node_fields<S>(post1, L, xk, yk, dr, u, w);
        fld[0][grp][k] = R(dr);
        fld[1][grp][k] = R(u);
        fld[2][grp][k] = R(w);
    }
    __syncthreads();
    if (act) {
        const R* drho = fld[0][grp];
        const R* ux = fld[1][grp];
        const R* uy = fld[2][grp];
        if (k < 4) {
            // end points relative to the support's centre node; thread k differentiates
            // along coordinate k of (X1.x, X1.y, X2.x, X2.y)
            using D1 = DN<R, 1>;
            const D1 c1x{R(X1.x - cx), {R(k == 0)}}, c1y{R(X1.y - cy), {R(k == 1)}};
            const D1 c2x{R(X2.x - cx), {R(k == 2)}}, c2y{R(X2.y - cy), {R(k == 3)}};
            const P2<D1> F = probe_traction<D1, R>(P2<D1>{c1x, c1y}, P2<D1>{c2x, c2y}, s, drho, ux, uy, R(L.nu));
            const double e = (double)(Fb[0] * F.x.d[0] + Fb[1] * F.y.d[0]);
            double* dst = k < 2 ? &xout[g1].x : &xout[g2].x;
            atomicAdd(dst + (k & 1), e);
        }
        // fields: dT/drho and dT/dG contracted with F_l-bar, for this thread's node
        const double sgn = s == 0 ? 1.0 : -1.0;
        const R nn[2] = {R(dy / len), R(-dx / len)};
        const R d0x = R(cx - Px), d0y = R(cy - Py);
        const ProbeVal<R> o = probe_eval<R, R>(d0x, d0y, drho, ux, uy);
        const R lsg = R(sgn * len), nu = R(L.nu);
        R rho_b = R(0), Gb[2][2];
        for (int a = 0; a < 2; a++) {
            R tt = -nn[a] / R(3);
            for (int b = 0; b < 2; b++) tt += nu * (o.G[a][b] + o.G[b][a]) * nn[b];
            rho_b += Fb[a] * lsg * tt;
        }
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) Gb[a][b] = lsg * o.rho * nu * (Fb[a] * nn[b] + Fb[b] * nn[a]);
        const Axis<R> ax = mls_axis<R>(d0x), ay = mls_axis<R>(d0y);
        const int a = k % 3, b = k / 3;
        // select rather than index with the thread's node (keeps the axes in registers)
        auto pick = [](const R (&v)[3], int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]); };
        const R qxa = pick(ax.q, a), hxa = pick(ax.h, a), gxa = pick(ax.g, a);
        const R qyb = pick(ay.q, b), hyb = pick(ay.h, b), gyb = pick(ay.g, b);
        const R phi = hxa * qyb + qxa * hyb - qxa * qyb;
        const R gx = gxa * qyb, gy = qxa * gyb;
        inject_fields(L, cell, (double)(phi * rho_b), (double)(Gb[0][0] * gx + Gb[0][1] * gy),
                      (double)(Gb[1][0] * gx + Gb[1][1] * gy), (double)R(u), (double)R(w), 1.0 + (double)R(dr), sbar,
                      gsx, gsy);
    }
    for (int o = 16; o > 0; o >>= 1) {
        gsx += __shfl_xor_sync(0xffffffffu, gsx, o);
        gsy += __shfl_xor_sync(0xffffffffu, gsy, o);
    }
    if ((threadIdx.x & 31) == 0 && (gsx != 0.0 || gsy != 0.0)) {
        atomicAdd(grad_g, gsx);
        atomicAdd(grad_g + 1, gsy);
    }
    if (!ok && k == 0) atomicOr(status, kStatSupport);
}

// Interpolation transpose (Eq. 8, velocity before any IB force) of U = I(s, X^n) at every
// vertex for a given U-bar: one thread per (vertex, support node). Adds to the population
// adjoint and dJ/dX^n (xout).
template <typename S>
__global__ void __launch_bounds__(kInterpThreads) k_adjd_interp(Lat L, const S* __restrict__ post,
                                                     const Shape* __restrict__ shp, int count, const double2* ubar,
                                                     double2* xout, double* sbar, double* grad_g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = t / 9, k = t - 9 * (t / 9);
    double gsx = 0.0, gsy = 0.0;
    if (v < count) {
        const double2 U = ubar[v];
        const int a = k % 3, b = k / 3;
        const Shape& s = shp[v];
        const int xk = wrapi(s.cx + a - 1, L.nx), yk = support_row(L, s.cy + b - 1);
        double drho, ux, uy;
        node_fields<S>(post, L, xk, yk, drho, ux, uy);
        const double uU = ux * U.x + uy * U.y;
        atomicAdd(&xout[v].x, s.px[b][a] * uU);
        atomicAdd(&xout[v].y, s.py[b][a] * uU);
        const double phi = s.phi[b][a];
        inject_fields(L, (long long)yk * L.nx + xk, 0.0, phi * U.x, phi * U.y, ux, uy, 1.0 + drho, sbar, gsx, gsy);
    }
    for (int o = 16; o > 0; o >>= 1) {
        gsx += __shfl_xor_sync(0xffffffffu, gsx, o);
        gsy += __shfl_xor_sync(0xffffffffu, gsy, o);
    }
    if ((threadIdx.x & 31) == 0 && (gsx != 0.0 || gsy != 0.0)) {
        atomicAdd(grad_g, gsx);
        atomicAdd(grad_g + 1, gsy);
    }
}

// DR3: spread transpose (with c_l), F_l = u_v - U and the start-up rule, one CTA per
// capsule. Completes dJ/dX^n in xout (except the U interpolation, added by the next
// kernel), writes U-bar (with Eq. 23's part, utb), the new u_v-bar and dJ/dX^{n-1}.
__global__ void __launch_bounds__(128) k_adjd_forcing(Lat L, Nodes nd, int max_n, const double2* Xn,
                                                      const double2* Flc, const Shape* __restrict__ shp,
                                                      const double* __restrict__ fbar, const double2* utb,
                                                      const int* age0, int nloc, double2* xout, double2* xm,
                                                      double2* ub, double2* u1b) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    const CapsuleParams P = nd.caps[blockIdx.x];
    if (P.n < 3 || P.n > max_n) return;
    const int n = P.n, off = P.off;
    const long long N = (long long)L.nx * L.ny;
    for (int v = threadIdx.x; v < n; v += blockDim.x) sm.X[v] = Xn[off + v];
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const int g = off + v;
        const Shape& s = shp[g];
        const double2 F = Flc[g];   // c_l F_l
        double cfx = 0.0, cfy = 0.0, gxv = 0.0, gyv = 0.0;
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int cell = support_cell(L, s, a, b);
                const double tx = fbar[cell], ty = fbar[N + cell];
                cfx += s.phi[b][a] * tx;
                cfy += s.phi[b][a] * ty;
                const double tF = tx * F.x + ty * F.y;
                gxv += s.px[b][a] * tF;
                gyv += s.py[b][a] * tF;
            }
        const double2 Xv = sm.X[v], Xl = sm.X[v == 0 ? n - 1 : v - 1], Xr = sm.X[v + 1 == n ? 0 : v + 1];
        const double ll = sqrt((Xv.x - Xl.x) * (Xv.x - Xl.x) + (Xv.y - Xl.y) * (Xv.y - Xl.y));
        const double lr = sqrt((Xr.x - Xv.x) * (Xr.x - Xv.x) + (Xr.y - Xv.y) * (Xr.y - Xv.y));
        const double cl = 0.5 * (ll + lr);
        // c-bar = F_l . (cF)-bar = (c F_l) . (cF)-bar / c;  F_l-bar = c (cF)-bar
        sm.sst[v] = (F.x * cfx + F.y * cfy) / cl;
        sm.ext[v] = make_double2(cl * cfx, cl * cfy);
        const double2 c = xout[g];
        sm.xd[v] = make_double2(c.x + gxv, c.y + gyv);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const int g = off + v;
        const int vl = v == 0 ? n - 1 : v - 1, vr = v + 1 == n ? 0 : v + 1;
        const double2 Xv = sm.X[v], Xl = sm.X[vl], Xr = sm.X[vr];
        const double dlx = Xv.x - Xl.x, dly = Xv.y - Xl.y, drx = Xr.x - Xv.x, dry = Xr.y - Xv.y;
        const double ll = sqrt(dlx * dlx + dly * dly), lr = sqrt(drx * drx + dry * dry);
        // c_u = (l_{u-1} + l_u)/2: X_v gets (d_{v-1}/l_{v-1})(c_v + c_{v-1})/2 - (d_v/l_v)(c_v + c_{v+1})/2
        const double wl = 0.5 * (sm.sst[v] + sm.sst[vl]) / ll, wr = 0.5 * (sm.sst[v] + sm.sst[vr]) / lr;
        double2 acc = sm.xd[v];
        acc.x += wl * dlx - wr * drx;
        acc.y += wl * dly - wr * dry;
        const double2 flb = sm.ext[v], xm1 = xm[g], ut = utb[g];
        if (age0[g] + nloc == 0) {
            // start-up: u_v := U (F_l = 0 whatever U is), X^{n-1} := X^n - U
            acc.x += xm1.x;
            acc.y += xm1.y;
            u1b[g] = make_double2(ut.x - xm1.x, ut.y - xm1.y);
            ub[g] = make_double2(0.0, 0.0);
            xm[g] = make_double2(0.0, 0.0);
        } else {
            u1b[g] = make_double2(ut.x - flb.x, ut.y - flb.y);
            ub[g] = flb;   // xm keeps dJ/dX^{n-1}
        }
        xout[g] = acc;
    }
}

inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace
}  // namespace lbmib

using namespace lbmib;

namespace {

// Workspace of one adjoint call.
struct AdjLayout {
    int K = 0, nseg = 0;
    size_t pb = 0, ckpt = 0;
    size_t tape_pops = 0, tape_X = 0, tape_flc = 0, age0 = 0, tape2_pops = 0, tape2_X = 0, tape2_flc = 0, age02 = 0, ckpts = 0, sbar[2]{}, fbar = 0,
           fib[3]{}, bbar[3]{}, xc = 0, xp = 0, xnew = 0, xb[2]{}, ub = 0, u1b = 0, u2b = 0, ftb = 0, fv = 0, fv1 = 0,
           shp = 0, shp1 = 0, grad = 0, J = 0, total = 0;
};

// The adjoint fields (population and force adjoints) are double in every storage mode:
// the body-force gradient sums them over every node and step.
size_t comp_bytes(lbmib_storage) { return sizeof(double); }

AdjLayout adj_layout(const lbmib_ctx* c, long long T, int K) {
    AdjLayout a;
    a.K = (int)(K >= T ? T : K);
    a.nseg = (int)((T + a.K - 1) / a.K);
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    const size_t cs = comp_bytes(c->cfg.storage);
    a.pb = up(9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage), kAlign);
    a.ckpt = a.pb + up(2 * N * sizeof(double), kAlign) + up(9 * M * sizeof(int) + 16, kAlign) +
             5 * up(M * sizeof(double2), kAlign) + up(M * sizeof(int), kAlign);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = up(o + bytes, kAlign); return r; };
    a.tape_pops = take((size_t)(a.K + 1) * a.pb);
    a.tape_X = take((size_t)(a.K + 1) * M * sizeof(double2));
    a.tape_flc = take((size_t)(a.K + 1) * M * sizeof(double2));   // Dynamic: c_l F_l per step
    a.age0 = take(M * sizeof(int));
    if (a.nseg > 1) {
        // a second tape: the recompute of one segment runs while the previous is reversed
        a.tape2_pops = take((size_t)(a.K + 1) * a.pb);
        a.tape2_X = take((size_t)(a.K + 1) * M * sizeof(double2));
        a.tape2_flc = take((size_t)(a.K + 1) * M * sizeof(double2));
        a.age02 = take(M * sizeof(int));
    }
    a.ckpts = take(a.nseg > 1 ? (size_t)(a.nseg + 1) * a.ckpt : 0);
    a.sbar[0] = take(9 * N * cs);
    a.sbar[1] = take(9 * N * cs);
    a.fbar = take(2 * N * cs);
    for (int r = 0; r < 3; r++) {
        a.fib[r] = take(2 * N * sizeof(double));
        a.bbar[r] = take(2 * N * sizeof(double));
    }
    a.xc = take(M * sizeof(double2));
    a.xb[0] = take(M * sizeof(double2));
    a.xb[1] = take(M * sizeof(double2));
    a.ub = take(M * sizeof(double2));
    a.u1b = take(M * sizeof(double2));
    a.u2b = take(M * sizeof(double2));
    a.ftb = take(M * sizeof(double2));
    a.xp = take(M * sizeof(double2));
    a.xnew = take(M * sizeof(double2));
    a.fv = take(M * sizeof(double2));
    a.fv1 = take(M * sizeof(double2));   // Kinematic: forces of the other step parity
    a.shp = take(M * sizeof(Shape));
    a.shp1 = take(M * sizeof(Shape));    // shapes of the other step parity
    a.grad = take((2 * c->caps.size() + 2) * sizeof(double));
    a.J = take(sizeof(double));
    a.total = o;
    return a;
}

// Device checkpoint of the context state (the content of lbmib_save_state).
lbmib_status ckpt_save(lbmib_ctx* c, char* dst, const AdjLayout& a) {
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    cudaStream_t s = c->stream;
    char* p = dst;
    LBMIB_CUDA(c, cudaMemcpyAsync(p, c->pops[c->cur], 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage),
                                  cudaMemcpyDeviceToDevice, s));
    p += a.pb;
    LBMIB_CUDA(c, cudaMemcpyAsync(p, c->fib[c->cur_fib], 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    p += up(2 * N * sizeof(double), kAlign);
    LBMIB_CUDA(c, cudaMemcpyAsync(p, &c->ctr->count[c->cur_fib], sizeof(int), cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(p + 16, c->list[c->cur_fib], 9 * M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    p += up(9 * M * sizeof(int) + 16, kAlign);
    double2* arrs[5] = {c->nd.X, c->nd.Xm1, c->nd.uv, c->nd.Fint, c->nd.Fext};
    for (auto* q : arrs) {
        LBMIB_CUDA(c, cudaMemcpyAsync(p, q, M * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        p += up(M * sizeof(double2), kAlign);
    }
    LBMIB_CUDA(c, cudaMemcpyAsync(p, c->nd.age, M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    return LBMIB_OK;
}

lbmib_status ckpt_load(lbmib_ctx* c, const char* src, const AdjLayout& a, cudaStream_t s) {
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    c->cur = 0;
    c->cur_fib = 0;
    const char* p = src;
    LBMIB_CUDA(c, cudaMemcpyAsync(c->pops[0], p, 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage),
                                  cudaMemcpyDeviceToDevice, s));
    p += a.pb;
    LBMIB_CUDA(c, cudaMemcpyAsync(c->fib[0], p, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemsetAsync(c->fib[1], 0, 2 * N * sizeof(double), s));
    p += up(2 * N * sizeof(double), kAlign);
    // list counts and claim stamps restart; the sticky status word is kept (a reverse
    // sweep may run beside this load and flag into it)
    LBMIB_CUDA(c, cudaMemsetAsync(&c->ctr->count[0], 0, 2 * sizeof(int), s));
    LBMIB_CUDA(c, cudaMemsetAsync(&c->ctr->step_stamp, 0, 2 * sizeof(int), s));
    LBMIB_CUDA(c, cudaMemcpyAsync(&c->ctr->count[0], p, sizeof(int), cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->list[0], p + 16, 9 * M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    p += up(9 * M * sizeof(int) + 16, kAlign);
    double2* arrs[5] = {c->nd.X, c->nd.Xm1, c->nd.uv, c->nd.Fint, c->nd.Fext};
    for (auto* q : arrs) {
        LBMIB_CUDA(c, cudaMemcpyAsync(q, p, M * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        p += up(M * sizeof(double2), kAlign);
    }
    LBMIB_CUDA(c, cudaMemcpyAsync(c->nd.age, p, M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemsetAsync(c->mark, 0, N * sizeof(int), s));
    return LBMIB_OK;
}

// Forward `len` steps from the context state, writing every step's populations into the
// tape (slot 0 = the starting state) and the vertex positions before every step.
lbmib_status tape_forward(lbmib_ctx* c, lbmib_scheme scheme, int len, char* w, const AdjLayout& a, cudaStream_t s) {
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    const size_t pbytes = 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage);
    char* tape = w + a.tape_pops;
    double2* tX = (double2*)(w + a.tape_X);
    LBMIB_CUDA(c, cudaMemcpyAsync(tape, c->pops[c->cur], pbytes, cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(w + a.age0, c->nd.age, M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    void* keep0 = c->pops[0];
    void* keep1 = c->pops[1];
    fork_ib(c, s);
    for (int k = 0; k < len; k++) {
        // positions before step k: after the previous node update, on the stream that runs it
        LBMIB_CUDA(c, cudaMemcpyAsync(tX + (size_t)k * M, c->nd.X, M * sizeof(double2), cudaMemcpyDeviceToDevice,
                                      ib_stream_of(c, s)));
        c->pops[0] = tape + (size_t)k * a.pb;
        c->pops[1] = tape + (size_t)(k + 1) * a.pb;
        if (scheme == LBMIB_DYNAMIC) c->nd.Flc = (double2*)(w + a.tape_flc) + (size_t)k * M;
        int cur = 0;
        enqueue_step(c, scheme, cur, c->cur_fib, s, false);
    }
    join_ib(c, s);
    c->nd.Flc = nullptr;
    c->pops[0] = keep0;
    c->pops[1] = keep1;
    LBMIB_CUDA(c, cudaMemcpyAsync(tX + (size_t)len * M, c->nd.X, M * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->pops[c->cur], tape + (size_t)len * a.pb, pbytes, cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaGetLastError());
    c->steps += len;
    return LBMIB_OK;
}

// Reverse sweep of one taped segment: global steps n0 + len - 1 down to n0.
// The spread of step n (membrane forces, shapes and spread at the taped X^n) depends on
// the tape alone, so while step n's interpolation, lattice and membrane transposes run,
// a side stream already spreads step n-1 into the other parity's forces and shapes and
// the third force buffer (cleared by step n+1's lattice transpose, whose completion it
// waits for); step n-1 waits for it before its interpolation transpose.
template <typename S>
lbmib_status reverse_segment(lbmib_ctx* c, long long n0, int len, char* w, const AdjLayout& a, cudaStream_t s) {
    cudaStream_t s2 = c->ib_stream;
    cudaEvent_t ev_prev = c->ev_adj[0], ev_spr = c->ev_adj[1];
    const Lat& L = c->L;
    const int ncaps = (int)c->caps.size();
    const int count = c->nd.count;
    const size_t M = (size_t)(count > 0 ? count : 1);
    const long long N = (long long)L.nx * L.ny;
    const size_t smem = ring_smem_bytes(c->max_n);
    double* grad = (double*)(w + a.grad);
    auto r3 = [](long long n) { return (int)(((n % 3) + 3) % 3); };
    double2* Fvs[2] = {(double2*)(w + a.fv), (double2*)(w + a.fv1)};     // forces at X^m in Fvs[m & 1]
    Shape* shps[2] = {(Shape*)(w + a.shp), (Shape*)(w + a.shp1)};       // shapes at X^m in shps[m & 1]
    auto spread = [&](long long m, int km, cudaStream_t q) {
        const double2* Xm = (const double2*)(w + a.tape_X) + (size_t)km * M;
        k_adj_spread<<<ncaps, 128, smem, q>>>(L, c->nd, Xm, c->max_n, Fvs[m & 1], shps[m & 1],
                                              (double*)(w + a.fib[r3(m)]));
    };
    for (int k = len - 1; k >= 0; k--) {
        const long long n = n0 + k;
        const int par = (int)(n & 1);
        const S* post0 = (const S*)(w + a.tape_pops + (size_t)k * a.pb);
        const S* post1 = (const S*)(w + a.tape_pops + (size_t)(k + 1) * a.pb);
        const double2* Xn = (const double2*)(w + a.tape_X) + (size_t)k * M;
        double* fib = (double*)(w + a.fib[r3(n)]);
        double* bbar = (double*)(w + a.bbar[par]);
        double* sb_in = (double*)(w + a.sbar[1 - par]);
        double* sb_out = (double*)(w + a.sbar[par]);
        double* fbar = (double*)(w + a.fbar);
        double2* xc = (double2*)(w + a.xc);
        double2* xp = (double2*)(w + a.xp);
        double2* xnew = (double2*)(w + a.xnew);
        if (ncaps > 0) {
            if (k == len - 1) spread(n, k, s);            // the segment's first reverse step
            else cudaStreamWaitEvent(s, ev_spr, 0);       // spread on the side stream last step
            if (k > 0) {
                cudaEventRecord(ev_prev, s);
                cudaStreamWaitEvent(s2, ev_prev, 0);
                spread(n - 1, k - 1, s2);
                cudaEventRecord(ev_spr, s2);
            }
            k_adj_interp<S><<<nblk(9LL * count, kInterpThreads), kInterpThreads, 0, s>>>(L, post1, fib, shps[par],
                                                                   (const int*)(w + a.age0), k, count, xc, xp, xnew,
                                                                   sb_in, bbar, grad + 2 * ncaps, &c->ctr->status);
        }
        k_adj_lattice<S><<<nblk(N, 256), 256, 0, s>>>(post0, L, sb_in, sb_out, fbar, fib,
                                                       (double*)(w + a.fib[r3(n + 1)]),
                                                       (double*)(w + a.bbar[1 - par]), grad + 2 * ncaps);
        if (ncaps > 0)
            k_adj_membrane<<<ncaps, 128, smem, s>>>(L, c->nd, Xn, c->max_n, Fvs[par], shps[par], fbar, bbar, xnew,
                                                       xc, ncaps, grad);
        c->launches += ncaps > 0 ? 4 : 1;
        LBMIB_CUDA(c, cudaGetLastError());
    }
    return LBMIB_OK;
}

// Reverse sweep of one taped Dynamic segment: global steps n0 + len - 1 down to n0.
template <typename S>
lbmib_status reverse_segment_dynamic(lbmib_ctx* c, long long n0, int len, char* w, const AdjLayout& a,
                                     cudaStream_t s) {
    const Lat& L = c->L;
    const int ncaps = (int)c->caps.size();
    const int count = c->nd.count;
    const size_t M = (size_t)(count > 0 ? count : 1);
    const long long N = (long long)L.nx * L.ny;
    const size_t smem = ring_smem_bytes(c->max_n);
    double* grad = (double*)(w + a.grad);
    auto r3 = [](long long n) { return (int)(((n % 3) + 3) % 3); };
    Shape* shps[2] = {(Shape*)(w + a.shp), (Shape*)(w + a.shp1)};   // shapes at X^m in shps[m & 1]
    double* fbar = (double*)(w + a.fbar);
    double2* xm = (double2*)(w + a.xp);
    double2* ub = (double2*)(w + a.ub);
    double2* u1b = (double2*)(w + a.u1b);
    double2* utb = (double2*)(w + a.u2b);   // adjoint of Eq. 23's tentative velocity
    const int* age0 = (const int*)(w + a.age0);
    // Two streams. The spread of step n-1 (taped positions and c_l F_l only) runs on a
    // side stream beside this step's chain, except at the segment's first reverse step,
    // whose own spread the chain needs; it waits for the previous reverse step, whose
    // lattice transpose clears the buffer it writes, and the next step's lattice
    // transpose, which reads it, waits for it.
    cudaStream_t s2 = c->ib_stream;
    cudaEvent_t ev_prev = c->ev_adj[0], ev_spr = c->ev_adj[1];
    bool pending = false;   // the side stream is spreading the step about to be reversed
    for (int k = len - 1; k >= 0; k--) {
        const long long n = n0 + k;
        const int par = (int)(n & 1);
        const S* post0 = (const S*)(w + a.tape_pops + (size_t)k * a.pb);
        const S* post1 = (const S*)(w + a.tape_pops + (size_t)(k + 1) * a.pb);
        const double2* Xn = (const double2*)(w + a.tape_X) + (size_t)k * M;
        const double2* flc = (const double2*)(w + a.tape_flc);
        double* fib_n = (double*)(w + a.fib[r3(n)]);
        double* fib_p = k > 0 ? (double*)(w + a.fib[r3(n - 1)]) : nullptr;
        double* sb_in = (double*)(w + a.sbar[1 - par]);
        double* sb_out = (double*)(w + a.sbar[par]);
        double2* xc = (double2*)(w + a.xb[1 - par]);
        double2* xout = (double2*)(w + a.xb[par]);
        Shape* shp = shps[par];
        const bool first = k == len - 1, side = !first && k > 0;
        if (ncaps > 0) {
            if (pending) cudaStreamWaitEvent(s, ev_spr, 0);   // this step's spread and shapes
            pending = false;
            if (first || side) {
                cudaStream_t q = first ? s : s2;
                if (side) {
                    cudaEventRecord(ev_prev, s);
                    cudaStreamWaitEvent(s2, ev_prev, 0);
                }
                k_adjd_spread<<<ncaps, 128, 0, q>>>(L, c->nd, c->max_n, Xn, k > 0 ? Xn - M : nullptr,
                                                    flc + (size_t)k * M, k > 0 ? flc + (size_t)(k - 1) * M : nullptr,
                                                    first ? fib_n : nullptr, fib_p, shp, shps[1 - par], first);
                if (side) {
                    cudaEventRecord(ev_spr, s2);
                    pending = true;
                }
            }
            k_adjd_update<<<ncaps, 128, smem, s>>>(c->nd, c->max_n, Xn, xc, xm, ub, xout, utb,
                                                   (double2*)(w + a.ftb), ncaps, grad);
            k_adjd_tract<S><<<nblk(2LL * count, kTractGroups), kTractThreads, 0, s>>>(
                L, c->nd, count, Xn, post1, (const double2*)(w + a.ftb), xout, sb_in, grad + 2 * ncaps,
                &c->ctr->status);
        }
        k_adj_lattice<S><<<nblk(N, 256), 256, 0, s>>>(post0, L, sb_in, sb_out, fbar, fib_n,
                                                       (double*)(w + a.fib[r3(n + 1)]), nullptr, grad + 2 * ncaps);
        if (ncaps > 0) {
            k_adjd_forcing<<<ncaps, 128, smem, s>>>(L, c->nd, c->max_n, Xn, flc + (size_t)k * M, shp, fbar, utb,
                                                    age0, k, xout, xm, ub, u1b);
            k_adjd_interp<S><<<nblk(9LL * count, kInterpThreads), kInterpThreads, 0, s>>>(L, post0, shp, count, u1b,
                                                                                          xout, sb_out,
                                                                                          grad + 2 * ncaps);
        }
        c->launches += ncaps > 0 ? (first || side ? 6 : 5) : 1;
        LBMIB_CUDA(c, cudaGetLastError());
    }
    return LBMIB_OK;
}

// Instantiated graphs of the segments of one adjoint call (destroyed with it).
struct SegmentGraph {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;   // kernels it runs
    int cur_fib = 0;          // force-buffer index after a recompute
};
struct SegmentGraphs {
    std::map<std::pair<int, int>, SegmentGraph> fwd;
    std::map<std::tuple<int, int, int>, SegmentGraph> rev;
    ~SegmentGraphs() {
        for (auto& kv : fwd) cudaGraphExecDestroy(kv.second.exec);
        for (auto& kv : rev) cudaGraphExecDestroy(kv.second.exec);
    }
};

// Events ordering the two tapes between the recompute and reverse streams.
struct Events {
    cudaEvent_t fdone[2]{}, rdone[2]{}, fork{};
    bool ok = true;
    Events() {
        for (cudaEvent_t* e : {&fdone[0], &fdone[1], &rdone[0], &rdone[1], &fork})
            ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    }
    ~Events() {
        for (cudaEvent_t e : {fdone[0], fdone[1], rdone[0], rdone[1], fork})
            if (e) cudaEventDestroy(e);
    }
};

// Capture what body(stream) enqueues on the context's capture stream into an
// instantiated graph. The capture is ended whatever body returns.
template <typename F>
lbmib_status capture_segment(lbmib_ctx* c, cudaGraphExec_t* exec, F&& body) {
    LBMIB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const lbmib_status st = body(c->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != LBMIB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture (adjoint segment)");
    const cudaError_t ei = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return cuda_fail(c, ei, "cudaGraphInstantiate (adjoint segment)");
    return LBMIB_OK;
}

}  // namespace

extern "C" {

size_t lbmib_adjoint_workspace_bytes(const lbmib_ctx* c, long long nsteps, int ckpt_every) {
    if (!c || nsteps < 1 || nsteps > (1LL << 30) || ckpt_every < 1) return 0;
    return adj_layout(c, nsteps, ckpt_every).total;
}

lbmib_status lbmib_adjoint(lbmib_ctx* c, long long nsteps, lbmib_scheme scheme, int ckpt_every, int objective,
                           int capsule, void* d_work, size_t work_bytes, double* J, double* grad) {
    if (!c) return LBMIB_ERR_ARG;
    if (nsteps < 1 || nsteps > (1LL << 30) || ckpt_every < 1 || !d_work || ((uintptr_t)d_work % kAlign) != 0 ||
        objective < 0 || objective > 2 || capsule < 0 || capsule >= (int)c->caps.size() || !grad)
        return fail(c, LBMIB_ERR_ARG, "lbmib_adjoint: invalid argument");
    if (scheme != LBMIB_KINEMATIC && scheme != LBMIB_DYNAMIC)
        return fail(c, LBMIB_ERR_ARG, "lbmib_adjoint: unknown scheme");
    if (c->rep_rc > 0.0 && c->caps.size() > 1)
        return fail(c, LBMIB_ERR_STATE, "lbmib_adjoint: the reverse sweep does not cover the capsule repulsion");
    if (c->L.inflow)
        return fail(c, LBMIB_ERR_STATE, "lbmib_adjoint: the reverse sweep does not cover the open-channel boundaries");
    if (c->nrigid > 0)
        return fail(c, LBMIB_ERR_STATE, "lbmib_adjoint: the reverse sweep does not cover rigid particles");
    const AdjLayout a = adj_layout(c, nsteps, ckpt_every);
    if (work_bytes < a.total) return fail(c, LBMIB_ERR_OOM, "lbmib_adjoint: workspace too small");
    lbmib_status st = device_status(c);
    if (st != LBMIB_OK) return st;
    if (c->max_n > 0) {
        const int sm_bytes = (int)ring_smem_bytes(c->max_n);
        cudaFuncSetAttribute(k_adj_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes);
        cudaFuncSetAttribute(k_adj_membrane, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes);
        cudaFuncSetAttribute(k_adjd_forcing, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes);
        cudaFuncSetAttribute(k_adjd_update, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes);
    }
    char* w = (char*)d_work;
    cudaStream_t s = c->stream;
    const int ncaps = (int)c->caps.size();
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    const size_t cs = comp_bytes(c->cfg.storage);
    // forward sweep
    if (a.nseg == 1) {
        st = tape_forward(c, scheme, (int)nsteps, w, a, s);
        if (st != LBMIB_OK) return st;
    } else {
        for (int j = 0; j < a.nseg; j++) {
            const long long len = std::min<long long>(a.K, nsteps - (long long)j * a.K);
            st = ckpt_save(c, w + a.ckpts + (size_t)j * a.ckpt, a);
            if (st == LBMIB_OK) st = lbmib_step(c, len, scheme);
            if (st != LBMIB_OK) return st;
        }
        st = ckpt_save(c, w + a.ckpts + (size_t)a.nseg * a.ckpt, a);
        if (st != LBMIB_OK) return st;
    }
    st = device_status(c);
    if (st != LBMIB_OK) return st;
    const long long steps_end = c->steps;
    // J and dJ/dX^T
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.xc, 0, M * sizeof(double2), s));
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.xp, 0, M * sizeof(double2), s));
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.xnew, 0, M * sizeof(double2), s));
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.ub, 0, M * sizeof(double2), s));
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.sbar[0], 0, 9 * N * cs, s));
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.sbar[1], 0, 9 * N * cs, s));
    for (int p = 0; p < 3; p++) {
        LBMIB_CUDA(c, cudaMemsetAsync(w + a.fib[p], 0, 2 * N * sizeof(double), s));
        LBMIB_CUDA(c, cudaMemsetAsync(w + a.bbar[p], 0, 2 * N * sizeof(double), s));
    }
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.grad, 0, (2 * ncaps + 2) * sizeof(double), s));
    // dJ/dX^T: the Kinematic sweep carries it in xc, the Dynamic one in the X-bar buffer of parity T
    double2* xT = scheme == LBMIB_KINEMATIC ? (double2*)(w + a.xc) : (double2*)(w + a.xb[nsteps & 1]);
    LBMIB_CUDA(c, cudaMemsetAsync(xT, 0, M * sizeof(double2), s));
    k_adj_objective<<<1, 256, 0, s>>>(c->nd, capsule, objective, xT, (double*)(w + a.J));
    c->launches++;
    LBMIB_CUDA(c, cudaGetLastError());
    // reverse sweep, segment by segment. With checkpoints, segment j - 1 is recomputed
    // into the other tape on a second stream while segment j is reversed (the reverse
    // sweep reads only its tape, the adjoint buffers and the constant capsule data; the
    // recompute only the context's working state and its tape). The recompute of a segment
    // depends only on its length and tape, and its reverse sweep on its length, tape and
    // first step modulo 6 (the parity and the modulo-3 rotation of the adjoint buffers):
    // each distinct shape is captured once into a CUDA graph and replayed for the segments
    // that share it.
    SegmentGraphs graphs;
    AdjLayout alt = a;
    alt.tape_pops = a.tape2_pops;
    alt.tape_X = a.tape2_X;
    alt.tape_flc = a.tape2_flc;
    alt.age0 = a.age02;
    auto tape_of = [&](int j) -> const AdjLayout& { return (j & 1) ? alt : a; };
    cudaStream_t sf = c->aux_stream;
    Events ev;
    if (!ev.ok) return fail(c, LBMIB_ERR_CUDA, "lbmib_adjoint: cudaEventCreateWithFlags failed");
    // how many segments share each shape: only a shape used more than once is captured
    std::map<std::pair<int, int>, int> fwd_uses;
    std::map<std::tuple<int, int, int>, int> rev_uses;
    for (int j = 0; j < a.nseg; j++) {
        const long long n0 = (long long)j * a.K;
        const int len = (int)std::min<long long>(a.K, nsteps - n0);
        fwd_uses[std::make_pair(len, j & 1)]++;
        rev_uses[std::make_tuple(len, (int)(n0 % 6), a.nseg > 1 ? (j & 1) : 0)]++;
    }
    auto recompute = [&](int j) -> lbmib_status {
        const int b = j & 1;
        const int len = (int)std::min<long long>(a.K, nsteps - (long long)j * a.K);
        if (j + 2 <= a.nseg - 1) LBMIB_CUDA(c, cudaStreamWaitEvent(sf, ev.rdone[b], 0));   // tape b free
        lbmib_status r = ckpt_load(c, w + a.ckpts + (size_t)j * a.ckpt, tape_of(j), sf);
        if (r != LBMIB_OK) return r;
        const std::pair<int, int> key(len, b);
        if (fwd_uses[key] <= 1) {   // a shape recomputed once is enqueued directly
            r = tape_forward(c, scheme, len, w, tape_of(j), sf);
            if (r != LBMIB_OK) return r;
            LBMIB_CUDA(c, cudaEventRecord(ev.fdone[b], sf));
            return LBMIB_OK;
        }
        auto it = graphs.fwd.find(key);
        if (it == graphs.fwd.end()) {
            SegmentGraph g;
            const long long launches0 = c->launches;
            r = capture_segment(c, &g.exec,
                                [&](cudaStream_t q) { return tape_forward(c, scheme, len, w, tape_of(j), q); });
            if (r != LBMIB_OK) return r;
            g.launches = c->launches - launches0;
            g.cur_fib = c->cur_fib;
            c->launches = launches0;
            c->steps -= len;   // the capture only recorded the steps
            it = graphs.fwd.emplace(key, g).first;
        }
        LBMIB_CUDA(c, cudaGraphLaunch(it->second.exec, sf));
        LBMIB_CUDA(c, cudaEventRecord(ev.fdone[b], sf));
        c->launches += it->second.launches;
        c->cur_fib = it->second.cur_fib;
        c->steps += len;
        return LBMIB_OK;
    };
    if (a.nseg > 1) {
        LBMIB_CUDA(c, cudaEventRecord(ev.fork, s));   // the objective and the cleared buffers
        LBMIB_CUDA(c, cudaStreamWaitEvent(sf, ev.fork, 0));
        st = recompute(a.nseg - 1);
        if (st != LBMIB_OK) return st;
    }
    for (int j = a.nseg - 1; j >= 0; j--) {
        const long long n0 = (long long)j * a.K;
        const int len = (int)std::min<long long>(a.K, nsteps - n0);
        const int b = j & 1;
        if (a.nseg > 1) {
            if (j > 0) {
                st = recompute(j - 1);
                if (st != LBMIB_OK) return st;
            }
            LBMIB_CUDA(c, cudaStreamWaitEvent(s, ev.fdone[b], 0));
        }
        const std::tuple<int, int, int> key(len, (int)(n0 % 6), a.nseg > 1 ? b : 0);
        const AdjLayout& t = a.nseg > 1 ? tape_of(j) : a;
        if (rev_uses[key] <= 1) {   // a shape reversed once is enqueued directly
            by_storage(c->cfg.storage, [&](auto tag) {
                using S = decltype(tag);
                st = scheme == LBMIB_KINEMATIC ? reverse_segment<S>(c, n0, len, w, t, s)
                                               : reverse_segment_dynamic<S>(c, n0, len, w, t, s);
            });
            if (st != LBMIB_OK) return st;
            if (a.nseg > 1) LBMIB_CUDA(c, cudaEventRecord(ev.rdone[b], s));
            continue;
        }
        auto it = graphs.rev.find(key);
        if (it == graphs.rev.end()) {
            SegmentGraph g;
            const long long launches0 = c->launches;
            st = capture_segment(c, &g.exec, [&](cudaStream_t q) {
                lbmib_status r = LBMIB_OK;
                by_storage(c->cfg.storage, [&](auto tag) {
                    using S = decltype(tag);
                    r = scheme == LBMIB_KINEMATIC ? reverse_segment<S>(c, n0, len, w, t, q)
                                                  : reverse_segment_dynamic<S>(c, n0, len, w, t, q);
                });
                return r;
            });
            if (st != LBMIB_OK) return st;
            g.launches = c->launches - launches0;
            c->launches = launches0;
            it = graphs.rev.emplace(key, g).first;
        }
        LBMIB_CUDA(c, cudaGraphLaunch(it->second.exec, s));
        if (a.nseg > 1) LBMIB_CUDA(c, cudaEventRecord(ev.rdone[b], s));
        c->launches += it->second.launches;
    }
    if (a.nseg > 1) {   // join the recompute stream before the context state is restored
        LBMIB_CUDA(c, cudaEventRecord(ev.fork, sf));
        LBMIB_CUDA(c, cudaStreamWaitEvent(s, ev.fork, 0));
    }
    if (a.nseg > 1) {
        st = ckpt_load(c, w + a.ckpts + (size_t)a.nseg * a.ckpt, a, s);
        if (st != LBMIB_OK) return st;
        c->steps = steps_end;
    }
    st = device_status(c);
    if (st != LBMIB_OK) return st;
    if (J) LBMIB_CUDA(c, cudaMemcpy(J, w + a.J, sizeof(double), cudaMemcpyDeviceToHost));
    LBMIB_CUDA(c, cudaMemcpy(grad, w + a.grad, (2 * ncaps + 2) * sizeof(double), cudaMemcpyDeviceToHost));
    return LBMIB_OK;
}

}  // extern "C"
