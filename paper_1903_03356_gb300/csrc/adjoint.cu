// Adjoint (reverse-mode derivative) of the Kinematic coupled step (Section 2.4, steps
// i-viii; Eq. 1-14, 25): gradients of a capsule objective J(X^T) (Taylor deformation D
// or centroid coordinate, Section 3.1) with respect to the membrane constants k_s, k_b
// of every capsule and the uniform body force g, over T steps from the current state.
//
// Forward step n (populations stored post-collision, s^n = pull(post^n) the streamed
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
#include <cstring>
#include <string>
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
// and the 2-D linear-basis shape function is phi_ab = h^x_a q^y_b + q^x_a h^y_b -
// q^x_a q^y_b (the closed-form MLS solve of the forward kernels written per axis).
// Evaluated on duals with d(d_a)/dX = -1 they give d(phi)/dX and d(phi)/dY.
// ---------------------------------------------------------------------------------
template <typename T>
struct Axis {
    T q[3], h[3];
};

template <typename T>
__device__ Axis<T> mls_axis(T d0) {
    T w[3], d[3];
    T s0 = T{0.0}, s1 = T{0.0};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        d[a] = d0 + double(a - 1);
        w[a] = dexp(-kMlsInvLen2 * (d[a] * d[a]));
        s0 = s0 + w[a];
        s1 = s1 + w[a] * d[a];
    }
    const T m = s1 / s0;
    T V = T{0.0};
#pragma unroll
    for (int a = 0; a < 3; a++) V = V + w[a] * ((d[a] - m) * (d[a] - m));
    Axis<T> r;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        r.q[a] = w[a] / s0;
        r.h[a] = r.q[a] - (m * w[a] * (d[a] - m)) / V;
    }
    return r;
}

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

template <typename T, typename GetX>
__device__ T ring_objective(int n, GetX X, int kind) {
    const P2<T> X0 = X(0);
    T s[6] = {T{0.0}, T{0.0}, T{0.0}, T{0.0}, T{0.0}, T{0.0}};
    for (int i = 0; i < n; i++) {
        const P2<T> a = X(i) - X0, b = X(i + 1 == n ? 0 : i + 1) - X0;
        const T c = a.x * b.y - b.x * a.y;
        s[0] = s[0] + c;
        s[1] = s[1] + (a.x + b.x) * c;
        s[2] = s[2] + (a.y + b.y) * c;
        s[3] = s[3] + (a.x * a.x + a.x * b.x + b.x * b.x) * c;
        s[4] = s[4] + (a.y * a.y + a.y * b.y + b.y * b.y) * c;
        s[5] = s[5] + (a.x * b.y + 2.0 * (a.x * a.y) + 2.0 * (b.x * b.y) + b.x * a.y) * c;
    }
    const T A = 0.5 * s[0];
    const T cx = s[1] / (6.0 * A), cy = s[2] / (6.0 * A);
    if (kind == kObjCentroidY) return cy + X0.y;
    if (kind == kObjCentroidX) return cx + X0.x;
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

// dJ/dX for every vertex of capsule `cap` (one dual evaluation per coordinate), J itself.
__global__ void k_adj_objective(Nodes nd, int cap, int kind, double2* xc, double* J) {
    const CapsuleParams P = nd.caps[cap];
    const int n = P.n;
    const double2* X = nd.X + P.off;
    for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) {
        const int vs = j >> 1, comp = j & 1;
        auto get = [&](int i) {
            const double2 p = X[i];
            return P2<Dual>{mk(p.x, i == vs && comp == 0 ? 1.0 : 0.0), mk(p.y, i == vs && comp == 1 ? 1.0 : 0.0)};
        };
        const Dual r = ring_objective<Dual>(n, get, kind);
        if (comp == 0) xc[P.off + vs].x = r.d;
        else xc[P.off + vs].y = r.d;
        if (j == 0) *J = r.v;
    }
}

// ---------------------------------------------------------------------------------
// R0: membrane forces at X^n (saved per vertex) and their spread into the force field.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_adj_spread(Lat L, Nodes nd, const double2* Xn, int max_n, double2* Fv,
                                                    double* fib) {
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
// vertex.
// ---------------------------------------------------------------------------------
template <typename S>
__global__ void k_adj_interp(Lat L, const S* __restrict__ post1, const double* __restrict__ fib, const double2* Xn,
                             const int* age0, int nloc, int count, double2* xc, double2* xp,
                             typename St<S>::C* sbar, double* bbar, double* grad_g, unsigned* status) {
    using C = typename St<S>::C;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    double gsx = 0.0, gsy = 0.0;
    if (v < count) {
        const bool first = age0[v] + nloc == 0;
        const double2 c = xc[v], p = xp[v];
        const double kU = first ? 1.0 : 2.0 / 3.0, kX = first ? 1.0 : 4.0 / 3.0;
        const double Ux = kU * c.x, Uy = kU * c.y;
        double ax = p.x + kX * c.x, ay = p.y + kX * c.y;
        xp[v] = first ? make_double2(0.0, 0.0) : make_double2(-c.x / 3.0, -c.y / 3.0);
        const Shape s = shape_with_derivatives(L, Xn[v].x, Xn[v].y);
        if (!s.ok) atomicOr(status, kStatSupport);
        const long long N = (long long)L.nx * L.ny;
#pragma unroll 1
        for (int b = 0; b < 3; b++)
#pragma unroll 1
            for (int a = 0; a < 3; a++) {
                const int xk = wrapi(s.cx + a - 1, L.nx), yk = support_row(L, s.cy + b - 1);
                const long long cell = (long long)yk * L.nx + xk;
                double q[9];
#pragma unroll
                for (int i = 0; i < 9; i++) q[i] = (double)pull<S>(post1, L, i, xk, yk);
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
                ax += s.px[b][a] * uU;
                ay += s.py[b][a] * uU;
                const double cf = s.phi[b][a] / rho;
#pragma unroll
                for (int i = 0; i < 9; i++) {
                    const double g = cf * ((ex(i) - ux) * Ux + (ey(i) - uy) * Uy);
                    atomicAdd(sbar + (long long)i * N + cell, (C)g);
                }
                atomicAdd(bbar + cell, 0.5 * cf * Ux);
                atomicAdd(bbar + N + cell, 0.5 * cf * Uy);
                gsx += 0.5 * cf * Ux;
                gsy += 0.5 * cf * Uy;
            }
        xc[v] = make_double2(ax, ay);
    }
    if (gsx != 0.0) atomicAdd(grad_g, gsx);
    if (gsy != 0.0) atomicAdd(grad_g + 1, gsy);
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
                                                     const typename St<S>::C* __restrict__ sb_in,
                                                     typename St<S>::C* __restrict__ sb_out,
                                                     typename St<S>::C* __restrict__ fbar,
                                                     const double* __restrict__ fib, double* fib_clear,
                                                     double* bbar_clear, double* grad_g) {
    using C = typename St<S>::C;
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
#pragma unroll
        for (int i = 0; i < 9; i++) s[i] = pull<S>(post0, L, i, x, y);
        const C Fx = C(L.gx + fib[node]), Fy = C(L.gy + fib[N + node]);
        C Fbx, Fby;
        collide_adjoint<C>(s, Fx, Fy, lat_c<C>(L.omega, L.omegaf), pb, sb, Fbx, Fby);
#pragma unroll
        for (int i = 0; i < 9; i++) sb_out[(long long)i * N + node] = sb[i];
        fbar[node] = Fbx;
        fbar[N + node] = Fby;
        fib_clear[node] = 0.0;
        fib_clear[N + node] = 0.0;
        bbar_clear[node] = 0.0;
        bbar_clear[N + node] = 0.0;
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

// ---------------------------------------------------------------------------------
// R3: spread and membrane transposes, one CTA per capsule.
//   F-bar_v = sum_k phi_k(X_v) fib-bar_k,  X-bar_v += sum_k grad phi_k (fib-bar_k . F_v)
//   X-bar_v += d/de F_v(X + e F-bar),      k_s-bar += F-bar . Fs,  k_b-bar += F-bar . Fb
// with fib-bar = (collision force adjoint) + (interpolation half-force adjoint).
// ---------------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(128) k_adj_membrane(Lat L, Nodes nd, const double2* Xn, int max_n,
                                                      const double2* Fv, const C* __restrict__ fbar,
                                                      const double* __restrict__ bbar, double2* xc, int ncaps,
                                                      double* grad) {
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
        const Shape s = shape_with_derivatives(L, sm.X[v].x, sm.X[v].y);
        const double2 F = Fv[off + v];
        double fbx = 0.0, fby = 0.0, gxv = 0.0, gyv = 0.0;
#pragma unroll
        for (int b = 0; b < 3; b++)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int cell = support_cell(L, s, a, b);
                const double tx = (double)fbar[cell] + bbar[cell];
                const double ty = (double)fbar[N + cell] + bbar[N + cell];
                fbx += s.phi[b][a] * tx;
                fby += s.phi[b][a] * ty;
                const double tF = tx * F.x + ty * F.y;
                gxv += s.px[b][a] * tF;
                gyv += s.py[b][a] * tF;
            }
        sm.ext[v] = make_double2(fbx, fby);   // F-bar of vertex v
        const double2 c = xc[off + v];
        xc[off + v] = make_double2(c.x + gxv, c.y + gyv);
    }
    __syncthreads();
    // area along the direction F-bar
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
        const double2 c = xc[off + v];
        xc[off + v] = make_double2(c.x + P.ks * Fs.x.d + P.kb * Fb.x.d + P.ka * Fa.x.d,
                                   c.y + P.ks * Fs.y.d + P.kb * Fb.y.d + P.ka * Fa.y.d);
    }
    block_reduce<2, false>(kk, sm.red);
    if (threadIdx.x == 0) {
        grad[cap] += kk[0];
        grad[ncaps + cap] += kk[1];
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
    size_t tape_pops = 0, tape_X = 0, age0 = 0, ckpts = 0, sbar[2]{}, fbar = 0, fib[2]{}, bbar[2]{}, xc = 0,
           xp = 0, fv = 0, grad = 0, J = 0, total = 0;
};

size_t comp_bytes(lbmib_storage s) { return s == LBMIB_FP64 ? 8 : 4; }

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
    a.age0 = take(M * sizeof(int));
    a.ckpts = take(a.nseg > 1 ? (size_t)(a.nseg + 1) * a.ckpt : 0);
    a.sbar[0] = take(9 * N * cs);
    a.sbar[1] = take(9 * N * cs);
    a.fbar = take(2 * N * cs);
    a.fib[0] = take(2 * N * sizeof(double));
    a.fib[1] = take(2 * N * sizeof(double));
    a.bbar[0] = take(2 * N * sizeof(double));
    a.bbar[1] = take(2 * N * sizeof(double));
    a.xc = take(M * sizeof(double2));
    a.xp = take(M * sizeof(double2));
    a.fv = take(M * sizeof(double2));
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

lbmib_status ckpt_load(lbmib_ctx* c, const char* src, const AdjLayout& a) {
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    cudaStream_t s = c->stream;
    c->cur = 0;
    c->cur_fib = 0;
    const char* p = src;
    LBMIB_CUDA(c, cudaMemcpyAsync(c->pops[0], p, 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage),
                                  cudaMemcpyDeviceToDevice, s));
    p += a.pb;
    LBMIB_CUDA(c, cudaMemcpyAsync(c->fib[0], p, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemsetAsync(c->fib[1], 0, 2 * N * sizeof(double), s));
    p += up(2 * N * sizeof(double), kAlign);
    LBMIB_CUDA(c, cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), s));
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
lbmib_status tape_forward(lbmib_ctx* c, lbmib_scheme scheme, int len, char* w, const AdjLayout& a) {
    cudaStream_t s = c->stream;
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    const size_t pbytes = 9 * (size_t)c->L.plane * storage_bytes(c->cfg.storage);
    char* tape = w + a.tape_pops;
    double2* tX = (double2*)(w + a.tape_X);
    LBMIB_CUDA(c, cudaMemcpyAsync(tape, c->pops[c->cur], pbytes, cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(w + a.age0, c->nd.age, M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    void* keep0 = c->pops[0];
    void* keep1 = c->pops[1];
    for (int k = 0; k < len; k++) {
        LBMIB_CUDA(c, cudaMemcpyAsync(tX + (size_t)k * M, c->nd.X, M * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        c->pops[0] = tape + (size_t)k * a.pb;
        c->pops[1] = tape + (size_t)(k + 1) * a.pb;
        int cur = 0;
        enqueue_step(c, scheme, cur, c->cur_fib, s, false);
    }
    c->pops[0] = keep0;
    c->pops[1] = keep1;
    LBMIB_CUDA(c, cudaMemcpyAsync(tX + (size_t)len * M, c->nd.X, M * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaMemcpyAsync(c->pops[c->cur], tape + (size_t)len * a.pb, pbytes, cudaMemcpyDeviceToDevice, s));
    LBMIB_CUDA(c, cudaGetLastError());
    c->steps += len;
    return LBMIB_OK;
}

// Reverse sweep of one taped segment: global steps n0 + len - 1 down to n0.
template <typename S>
lbmib_status reverse_segment(lbmib_ctx* c, long long n0, int len, char* w, const AdjLayout& a) {
    using C = typename St<S>::C;
    cudaStream_t s = c->stream;
    const Lat& L = c->L;
    const int ncaps = (int)c->caps.size();
    const int count = c->nd.count;
    const size_t M = (size_t)(count > 0 ? count : 1);
    const long long N = (long long)L.nx * L.ny;
    const size_t smem = ring_smem_bytes(c->max_n);
    double* grad = (double*)(w + a.grad);
    for (int k = len - 1; k >= 0; k--) {
        const int par = (int)((n0 + k) & 1);
        const S* post0 = (const S*)(w + a.tape_pops + (size_t)k * a.pb);
        const S* post1 = (const S*)(w + a.tape_pops + (size_t)(k + 1) * a.pb);
        const double2* Xn = (const double2*)(w + a.tape_X) + (size_t)k * M;
        double* fib = (double*)(w + a.fib[par]);
        double* bbar = (double*)(w + a.bbar[par]);
        C* sb_in = (C*)(w + a.sbar[1 - par]);
        C* sb_out = (C*)(w + a.sbar[par]);
        C* fbar = (C*)(w + a.fbar);
        double2* Fv = (double2*)(w + a.fv);
        double2* xc = (double2*)(w + a.xc);
        double2* xp = (double2*)(w + a.xp);
        if (ncaps > 0) {
            k_adj_spread<<<ncaps, 128, smem, s>>>(L, c->nd, Xn, c->max_n, Fv, fib);
            k_adj_interp<S><<<nblk(count, 128), 128, 0, s>>>(L, post1, fib, Xn, (const int*)(w + a.age0), k, count,
                                                             xc, xp, sb_in, bbar, grad + 2 * ncaps,
                                                             &c->ctr->status);
        }
        k_adj_lattice<S><<<nblk(N, 256), 256, 0, s>>>(post0, L, sb_in, sb_out, fbar, fib,
                                                       (double*)(w + a.fib[1 - par]),
                                                       (double*)(w + a.bbar[1 - par]), grad + 2 * ncaps);
        if (ncaps > 0)
            k_adj_membrane<C><<<ncaps, 128, smem, s>>>(L, c->nd, Xn, c->max_n, Fv, fbar, bbar, xc, ncaps, grad);
        c->launches += ncaps > 0 ? 4 : 1;
        LBMIB_CUDA(c, cudaGetLastError());
    }
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
    if (scheme != LBMIB_KINEMATIC)
        return fail(c, LBMIB_ERR_ARG, "lbmib_adjoint: the reverse sweep covers the Kinematic scheme");
    const AdjLayout a = adj_layout(c, nsteps, ckpt_every);
    if (work_bytes < a.total) return fail(c, LBMIB_ERR_OOM, "lbmib_adjoint: workspace too small");
    lbmib_status st = device_status(c);
    if (st != LBMIB_OK) return st;
    if (c->max_n > 0) {
        const int sm_bytes = (int)ring_smem_bytes(c->max_n);
        cudaFuncSetAttribute(k_adj_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes);
        cudaFuncSetAttribute(k_adj_membrane<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes);
        cudaFuncSetAttribute(k_adj_membrane<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_bytes);
    }
    char* w = (char*)d_work;
    cudaStream_t s = c->stream;
    const int ncaps = (int)c->caps.size();
    const size_t N = (size_t)c->cfg.nx * c->cfg.ny;
    const size_t M = (size_t)(c->nd.count > 0 ? c->nd.count : 1);
    const size_t cs = comp_bytes(c->cfg.storage);
    // forward sweep
    if (a.nseg == 1) {
        st = tape_forward(c, scheme, (int)nsteps, w, a);
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
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.sbar[0], 0, 9 * N * cs, s));
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.sbar[1], 0, 9 * N * cs, s));
    for (int p = 0; p < 2; p++) {
        LBMIB_CUDA(c, cudaMemsetAsync(w + a.fib[p], 0, 2 * N * sizeof(double), s));
        LBMIB_CUDA(c, cudaMemsetAsync(w + a.bbar[p], 0, 2 * N * sizeof(double), s));
    }
    LBMIB_CUDA(c, cudaMemsetAsync(w + a.grad, 0, (2 * ncaps + 2) * sizeof(double), s));
    k_adj_objective<<<1, 256, 0, s>>>(c->nd, capsule, objective, (double2*)(w + a.xc), (double*)(w + a.J));
    c->launches++;
    LBMIB_CUDA(c, cudaGetLastError());
    // reverse sweep, segment by segment
    for (int j = a.nseg - 1; j >= 0; j--) {
        const long long n0 = (long long)j * a.K;
        const int len = (int)std::min<long long>(a.K, nsteps - n0);
        if (a.nseg > 1) {
            st = ckpt_load(c, w + a.ckpts + (size_t)j * a.ckpt, a);
            if (st == LBMIB_OK) st = tape_forward(c, scheme, len, w, a);
            if (st != LBMIB_OK) return st;
        }
        by_storage(c->cfg.storage, [&](auto tag) {
            using S = decltype(tag);
            if (st == LBMIB_OK) st = reverse_segment<S>(c, n0, len, w, a);
        });
        if (st != LBMIB_OK) return st;
    }
    if (a.nseg > 1) {
        st = ckpt_load(c, w + a.ckpts + (size_t)a.nseg * a.ckpt, a);
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
