// Device-side building blocks of the LBM-IB library (sm_103a).
//
// Method: Coclite et al., arXiv:1903.03356. D2Q9 BGK with a body-force term
// (Section 2.1-2.2, Eq. 1-7), MLS transfer (Eq. 8-9), membrane forces (Eq. 10-16).
//
// Lattice storage: structure of arrays, population-major: plane i holds ny rows of
// `pitch` elements (pitch = nx rounded up to 128 bytes). The stored value of population
// i is the POST-collision value minus its rest weight w_i (shifted storage), so a step
// is a pull: node x gathers population i from x - e_i, collides, and writes its own
// slot. A population whose source lies beyond a wall is the node's own outgoing
// population in the opposite direction, corrected by -6 w_j (e_j . u_w) (half-way
// bounce-back with the reference density rho_0 = 1).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmib {

// ---------------------------------------------------------------------------------
// D2Q9 velocity set (Eq. 3) and weights (Section 2.1)
// ---------------------------------------------------------------------------------
__host__ __device__ constexpr int ex(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
template <typename C>
__host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp axis");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp diag");

// Lattice description passed by value to every kernel.
struct Lat {
    int nx, ny;
    int pitch;            // elements per stored row
    int walls;            // 1: bounce-back walls at y = -1/2 and y = ny - 1/2
    long long plane;      // elements per population plane (ny * pitch)
    double tau, omega;    // relaxation time and 1/tau
    double ub, ut;        // wall x-velocities (bottom, top)
    double gx, gy;        // uniform body-force density
    float scale, inv_scale;  // FP16 storage scale (1 for other storages)
    double nu;            // kinematic viscosity (tau - 1/2)/3
    // float copies for single-precision kernels (a double-to-float conversion in every
    // thread would occupy GB300's narrow FP64 pipe)
    float gxf, gyf, omegaf, ubf, utf;
    // open channel (0: periodic in x; the boundary data travel in OpenBC). Placed in the
    // tail padding: the size of this struct, and with it the register allocation of the
    // lattice kernel, stays as it was.
    int inflow;
};

// Open channel: Zou-He known-velocity inlet at column 0 with x-velocity u_in[y] (device,
// ny values), known-density outlet at column nx - 1. Passed only to the kernels whose
// results at the open columns are used (supports of markers and probes stay off them).
struct OpenBC {
    const double* u_in;
    double drho_out;      // outlet density - 1
    float drho_outf;
};

// Lattice constant in the compute type C.
template <typename C>
__device__ __forceinline__ C lat_c(double d, float f) {
    if constexpr (sizeof(C) == 8) return d;
    else return f;
}

// ---------------------------------------------------------------------------------
// Storage traits: type S stored, type C computed in. ld goes through the read-only
// (non-coherent) path and is only for data the kernel never writes; ldc is a plain
// load for kernels that read populations they wrote earlier in the same launch.
// ---------------------------------------------------------------------------------
template <typename S>
struct St;
template <>
struct St<double> {
    using C = double;
    static __device__ __forceinline__ double ld(const double* p, const Lat&) { return __ldg(p); }
    static __device__ __forceinline__ double ldc(const double* p, const Lat&) { return *p; }
    static __device__ __forceinline__ void st(double* p, double v, const Lat&) { *p = v; }
};
template <>
struct St<float> {
    using C = float;
    static __device__ __forceinline__ float ld(const float* p, const Lat&) { return __ldg(p); }
    static __device__ __forceinline__ float ldc(const float* p, const Lat&) { return *p; }
    static __device__ __forceinline__ void st(float* p, float v, const Lat&) { *p = v; }
};
template <>
struct St<__half> {
    using C = float;
    // the unscaling is never fused with a following wall correction, so that every
    // kernel rounds a loaded FP16 population the same way
    static __device__ __forceinline__ float ld(const __half* p, const Lat& L) {
        return __fmul_rn(__half2float(__ldg(p)), L.inv_scale);
    }
    static __device__ __forceinline__ float ldc(const __half* p, const Lat& L) {
        return __fmul_rn(__half2float(*p), L.inv_scale);
    }
    static __device__ __forceinline__ void st(__half* p, float v, const Lat& L) {
        *p = __float2half_rn(v * L.scale);
    }
};

// Single-precision storage seen by the immersed-boundary kernels that compute in double
// (LBMIB_OPT_IB_FP64): the same 4- and 2-byte words, loaded as the storage type and then
// widened, so that those kernels keep their gathers in storage precision and do the MLS
// solve, the membrane and traction forces and the node update in FP64.
struct f32w {
    float v;
};
struct f16w {
    __half v;
};
static_assert(sizeof(f32w) == sizeof(float) && sizeof(f16w) == sizeof(__half), "storage views keep the word size");
template <>
struct St<f32w> {
    using C = double;
    static __device__ __forceinline__ double ld(const f32w* p, const Lat&) { return (double)__ldg(&p->v); }
    static __device__ __forceinline__ double ldc(const f32w* p, const Lat&) { return (double)p->v; }
    static __device__ __forceinline__ void st(f32w* p, double v, const Lat&) { p->v = (float)v; }
};
template <>
struct St<f16w> {
    using C = double;
    static __device__ __forceinline__ double ld(const f16w* p, const Lat& L) {
        return (double)__fmul_rn(__half2float(__ldg(&p->v)), L.inv_scale);
    }
    static __device__ __forceinline__ double ldc(const f16w* p, const Lat& L) {
        return (double)__fmul_rn(__half2float(p->v), L.inv_scale);
    }
    static __device__ __forceinline__ void st(f16w* p, double v, const Lat& L) {
        p->v = __float2half_rn((float)v * L.scale);
    }
};

__device__ __forceinline__ int wrapi(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Pre-collision population i at node (x, y) of the step that reads `src` (Eq. 1, left
// side): the pull of the post-collision population from x - e_i, or the wall reflection
// (periodic x only: the open columns of an open channel need pull_all).
// NC selects the read-only load path (src not written during the launch).
template <typename S, bool NC = true>
__device__ __forceinline__ typename St<S>::C pull(const S* __restrict__ src, const Lat& L, int i,
                                                  int x, int y) {
    using C = typename St<S>::C;
    int ys = y - ey(i);
    auto ld = [&](const S* p) { return NC ? St<S>::ld(p, L) : St<S>::ldc(p, L); };
    if (L.walls && (ys < 0 || ys >= L.ny)) {
        const int j = opp(i);
        const C uw = ys < 0 ? lat_c<C>(L.ub, L.ubf) : lat_c<C>(L.ut, L.utf);
        return ld(src + (long long)j * L.plane + (long long)y * L.pitch + x) - C(6) * wgt<C>(j) * C(ex(j)) * uw;
    }
    ys = wrapi(ys, L.ny);
    const int xs = wrapi(x - ex(i), L.nx);
    return ld(src + (long long)i * L.plane + (long long)ys * L.pitch + xs);
}

// Zou-He closure of an open column (inlet x = 0, outlet x = nx - 1) on the shifted
// pre-collision populations s of node (x, y): the three populations that enter from
// outside the lattice are rebuilt so that the node has velocity (u_in(y), 0) (inlet) or
// density rho_out and zero y-velocity (outlet), the non-equilibrium part bounced back
// along the normal and the tangential one shared by the diagonals. The known momentum is
// rho u - F/2 with F the uniform force (supports stay off the open columns). Explicit
// form of the closure in shifted variables (the rest weights cancel pairwise).
template <typename C>
__device__ __forceinline__ void open_column(C (&s)[9], const Lat& L, const OpenBC& ob, int x, int y) {
    const C Fx = lat_c<C>(L.gx, L.gxf), Fy = lat_c<C>(L.gy, L.gyf);
    const C jy = C(-0.5) * Fy;
    const C t = C(0.5) * (s[2] - s[4]);
    if (x == 0) {
        const C u = C(ob.u_in[y]);
        // rho (1 - u) = 1 + s0 + s2 + s4 + 2 (s3 + s6 + s7) - Fx/2
        const C known = (s[0] + s[2] + s[4]) + C(2) * (s[3] + s[6] + s[7]);
        const C drho = (known - C(0.5) * Fx + u) / (C(1) - u);
        const C jx = (C(1) + drho) * u - C(0.5) * Fx;
        s[1] = s[3] + C(2.0 / 3.0) * jx;
        s[5] = s[7] - t + jx * C(1.0 / 6.0) + C(0.5) * jy;
        s[8] = s[6] + t + jx * C(1.0 / 6.0) - C(0.5) * jy;
    } else {
        // mass fixes the entering populations' sum, x-momentum follows
        const C jx = ((s[0] + s[2] + s[4]) + C(2) * (s[1] + s[5] + s[8])) - lat_c<C>(ob.drho_out, ob.drho_outf);
        s[3] = s[1] - C(2.0 / 3.0) * jx;
        s[7] = s[5] + t - jx * C(1.0 / 6.0) - C(0.5) * jy;
        s[6] = s[8] - t - jx * C(1.0 / 6.0) + C(0.5) * jy;
    }
}

// All nine pre-collision populations of node (x, y), as pull() but with the neighbour
// coordinates formed by comparisons instead of the periodic wrap's integer division,
// and every load issued before any is used, and, given the open-channel data ob, the
// Zou-He closure on the open columns. NC as for pull().
template <typename S, bool NC = true>
__device__ __forceinline__ void pull_all(const S* __restrict__ src, const Lat& L, int x, int y,
                                         typename St<S>::C (&s)[9], const OpenBC* ob = nullptr) {
    using C = typename St<S>::C;
    const int xm = x == 0 ? L.nx - 1 : x - 1, xp = x + 1 == L.nx ? 0 : x + 1;
    const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y + 1 == L.ny ? 0 : y + 1;
    const bool lo = L.walls && y == 0, hi = L.walls && y == L.ny - 1;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const bool bounce = (ey(i) > 0 && lo) || (ey(i) < 0 && hi);
        const int sx = ex(i) > 0 ? xm : (ex(i) < 0 ? xp : x);
        const int sy = ey(i) > 0 ? ym : (ey(i) < 0 ? yp : y);
        const S* p = src + (long long)(bounce ? opp(i) : i) * L.plane + (long long)(bounce ? y : sy) * L.pitch +
                     (bounce ? x : sx);
        s[i] = NC ? St<S>::ld(p, L) : St<S>::ldc(p, L);
    }
#pragma unroll
    for (int i = 0; i < 9; i++) {
        if ((ey(i) > 0 && lo) || (ey(i) < 0 && hi)) {
            const int j = opp(i);
            const C uw = ey(i) > 0 ? lat_c<C>(L.ub, L.ubf) : lat_c<C>(L.ut, L.utf);
            s[i] -= C(6) * wgt<C>(j) * C(ex(j)) * uw;
        }
    }
    // open channel: what the periodic wrap brought across the inlet or outlet is replaced
    if (ob && L.inflow && (x == 0 || x == L.nx - 1)) open_column<C>(s, L, *ob, x, y);
}

// Density deviation, momentum (Eq. 6-7 without the force) of shifted populations.
template <typename C>
__device__ __forceinline__ void moments(const C s[9], C& drho, C& mx, C& my) {
    drho = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + s[8];
    mx = (s[1] - s[3]) + (s[5] - s[6]) + (s[8] - s[7]);
    my = (s[2] - s[4]) + (s[5] + s[6]) - (s[7] + s[8]);
}

// BGK collision with the Guo forcing term (Eq. 4-5) on shifted populations, in place.
// F is the total force density at the node. Returns u^2 for the stability check.
// Opposite directions i and opp(i) see e.u and e.F change sign and their squares and
// products not, so the shifted equilibrium and the Guo term split into a part even and
// a part odd in e, computed once per pair:
//   f_eq - w = w (drho + rho (4.5 (e.u)^2 - 1.5 u^2))  +/-  3 w rho (e.u)
//   Guo term = (1 - 1/2tau) w (9 (e.u)(e.F) - 3 u.F)    +/-  3 (1 - 1/2tau) w (e.F)
template <typename C>
__device__ __forceinline__ C collide(C s[9], C Fx, C Fy, C omega) {
    C drho, mx, my;
    moments<C>(s, drho, mx, my);
    const C rho = C(1) + drho;
    const C inv = C(1) / rho;
    const C ux = (mx + C(0.5) * Fx) * inv;
    const C uy = (my + C(0.5) * Fy) * inv;
    const C usq = ux * ux + uy * uy;
    const C u15 = C(1.5) * usq;
    const C fpre = C(1) - C(0.5) * omega;   // 1 - 1/(2 tau)
    const C uF3 = C(3) * (ux * Fx + uy * Fy);
    const C keep = C(1) - omega;
    // rest population: even parts only
    s[0] = keep * s[0] + wgt<C>(0) * (omega * (drho - rho * u15) - fpre * uF3);
    // the pairs (1, 3), (2, 4), (5, 7), (6, 8): i has e = (ex, ey), opp(i) has -e
#pragma unroll
    for (int i : {1, 2, 5, 6}) {
        const int j = opp(i);
        const C eu = C(ex(i)) * ux + C(ey(i)) * uy;
        const C eF = C(ex(i)) * Fx + C(ey(i)) * Fy;
        const C w = wgt<C>(i);
        const C even = w * (omega * (drho + rho * (C(4.5) * eu * eu - u15)) + fpre * (C(9) * eu * eF - uF3));
        const C odd = C(3) * w * (omega * rho * eu + fpre * eF);
        s[i] = keep * s[i] + (even + odd);
        s[j] = keep * s[j] + (even - odd);
    }
    if constexpr (sizeof(C) < 8) {
        // Single precision: rounding inside the collision would break the exact
        // conservation of mass and momentum, and the lattice has no restoring force for
        // those errors, so they would accumulate step after step. Populations 1, 2 and
        // 0 are therefore set from the exact post-collision moments (sum s = drho,
        // sum s e = m + F); in exact arithmetic this changes nothing.
        s[1] = s[3] + ((mx + Fx) - ((s[5] - s[6]) + (s[8] - s[7])));
        s[2] = s[4] + ((my + Fy) - ((s[5] + s[6]) - (s[7] + s[8])));
        s[0] = drho - (((s[1] + s[2]) + (s[3] + s[4])) + ((s[5] + s[6]) + (s[7] + s[8])));
    }
    return usq;
}

// The forced post-collision populations of a node from its unforced ones (in place).
// collide() is keep * s + E(drho, u, F), where only E, the equilibrium and Guo parts,
// depends on the force, and the unforced collision kept the mass and added g to the
// momentum: so drho = sum s* and m = sum s* e - g, and the force g + f_ib gives
// s* + E(drho, u', F) - E(drho, u, g), u = (m + g/2)/rho, u' = (m + F/2)/rho, with
// rounding apart the populations collide() gives for F. (gx, gy) is the uniform force the
// unforced collision used, (Fx, Fy) the total. Returns u'^2 for the stability check.
template <typename C>
__device__ __forceinline__ C force_node(C s[9], C gx, C gy, C Fx, C Fy, C omega) {
    C drho, px, py;
    moments<C>(s, drho, px, py);
    const C mx = px - gx, my = py - gy;
    const C rho = C(1) + drho;
    const C inv = C(1) / rho;
    const C ux0 = (mx + C(0.5) * gx) * inv, uy0 = (my + C(0.5) * gy) * inv;
    const C ux = (mx + C(0.5) * Fx) * inv, uy = (my + C(0.5) * Fy) * inv;
    const C usq0 = ux0 * ux0 + uy0 * uy0, usq = ux * ux + uy * uy;
    const C fpre = C(1) - C(0.5) * omega;
    const C uF30 = C(3) * (ux0 * gx + uy0 * gy), uF3 = C(3) * (ux * Fx + uy * Fy);
    s[0] += wgt<C>(0) * (omega * rho * (C(1.5) * (usq0 - usq)) - fpre * (uF3 - uF30));
#pragma unroll
    for (int i : {1, 2, 5, 6}) {
        const int j = opp(i);
        const C eu0 = C(ex(i)) * ux0 + C(ey(i)) * uy0, eu = C(ex(i)) * ux + C(ey(i)) * uy;
        const C eg = C(ex(i)) * gx + C(ey(i)) * gy, eF = C(ex(i)) * Fx + C(ey(i)) * Fy;
        const C w = wgt<C>(i);
        const C even = w * (omega * rho * (C(4.5) * (eu * eu - eu0 * eu0) - C(1.5) * (usq - usq0)) +
                            fpre * ((C(9) * eu * eF - uF3) - (C(9) * eu0 * eg - uF30)));
        const C odd = C(3) * w * (omega * rho * (eu - eu0) + fpre * (eF - eg));
        s[i] += even + odd;
        s[j] += even - odd;
    }
    if constexpr (sizeof(C) < 8) {   // the conservation reset of collide()
        s[1] = s[3] + ((mx + Fx) - ((s[5] - s[6]) + (s[8] - s[7])));
        s[2] = s[4] + ((my + Fy) - ((s[5] + s[6]) - (s[7] + s[8])));
        s[0] = drho - (((s[1] + s[2]) + (s[3] + s[4])) + ((s[5] + s[6]) + (s[7] + s[8])));
    }
    return usq;
}

// Two single-precision lanes in one instruction (packed FP32 add, sub, mul and fma of
// sm_100 and later): the single-precision lattice kernels update lattice nodes in pairs.
// Each lane rounds as the scalar instruction would.
struct F2 {
    float x, y;
};
__device__ __forceinline__ F2 f2(float a) { return F2{a, a}; }
#define LBMIB_F2_BINARY(NAME, INSTR)                                                               \
    __device__ __forceinline__ F2 NAME(F2 a, F2 b) {                                               \
        F2 r;                                                                                      \
        asm("{.reg .b64 ra, rb, rd;\n\t"                                                           \
            "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" INSTR " rd, ra, rb;\n\t"           \
            "mov.b64 {%0, %1}, rd;}"                                                               \
            : "=f"(r.x), "=f"(r.y)                                                                 \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                             \
        return r;                                                                                  \
    }
LBMIB_F2_BINARY(operator+, "add.rn.f32x2")
LBMIB_F2_BINARY(operator-, "sub.rn.f32x2")
LBMIB_F2_BINARY(operator*, "mul.rn.f32x2")
#undef LBMIB_F2_BINARY
// a * b + c, one rounding per lane
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 r;
    asm("{.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// collide<float> (Eq. 4-5, the direction-pair form and the single-precision
// conservation reset) on two nodes at once, lane by lane; the same uniform force at both.
// Returns u^2 of each node.
__device__ __forceinline__ F2 collide2(F2 s[9], float Fx, float Fy, float omega) {
    const F2 drho = (((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]))) + s[8];
    const F2 mx = ((s[1] - s[3]) + (s[5] - s[6])) + (s[8] - s[7]);
    const F2 my = ((s[2] - s[4]) + (s[5] + s[6])) - (s[7] + s[8]);
    const F2 rho = f2(1.0f) + drho;
    const F2 inv = F2{1.0f / rho.x, 1.0f / rho.y};
    const F2 ux = (mx + f2(0.5f * Fx)) * inv;
    const F2 uy = (my + f2(0.5f * Fy)) * inv;
    const F2 usq = fma2(ux, ux, uy * uy);
    const F2 u15 = f2(1.5f) * usq;
    const float fpre = 1.0f - 0.5f * omega;
    const F2 uF3 = f2(3.0f) * fma2(ux, f2(Fx), uy * f2(Fy));
    const F2 keep = f2(1.0f - omega), om = f2(omega);
    s[0] = fma2(keep, s[0], f2(4.0f / 9.0f) * (om * (drho - rho * u15) - f2(fpre) * uF3));
#pragma unroll
    for (int i : {1, 2, 5, 6}) {
        const int j = opp(i);
        const F2 eu = i == 1 ? ux : (i == 2 ? uy : (i == 5 ? ux + uy : uy - ux));
        const float eF = float(ex(i)) * Fx + float(ey(i)) * Fy;
        const float w = wgt<float>(i);
        const F2 even = f2(w) * fma2(om, fma2(rho, fma2(f2(4.5f) * eu, eu, f2(0.0f) - u15), drho),
                                     f2(fpre) * (f2(9.0f * eF) * eu - uF3));
        const F2 odd = f2(3.0f * w) * fma2(om * rho, eu, f2(fpre * eF));
        s[i] = fma2(keep, s[i], even + odd);
        s[j] = fma2(keep, s[j], even - odd);
    }
    // conservation reset (see collide<float>)
    s[1] = s[3] + ((mx + f2(Fx)) - ((s[5] - s[6]) + (s[8] - s[7])));
    s[2] = s[4] + ((my + f2(Fy)) - ((s[5] + s[6]) - (s[7] + s[8])));
    s[0] = drho - (((s[1] + s[2]) + (s[3] + s[4])) + ((s[5] + s[6]) + (s[7] + s[8])));
    return usq;
}

// ---------------------------------------------------------------------------------
// Moving least squares (Eq. 8-9): 3x3 support centred on the nearest node, weights
// exp(-(r/alpha)^2), r = |x - x_k| / r_w, r_w = 2.6, alpha = 0.3, linear basis.
//
// The weight factorises, W_k = exp(-dx_a^2 / L^2) exp(-dy_b^2 / L^2) with L = r_w alpha,
// and the support is the tensor grid of three x and three y offsets. In the basis
// (1, dx - mx, dy - my), with mx, my the weighted mean offsets, every off-diagonal entry
// of the moment matrix A = sum W p p^T is a product containing sum_a wx_a (dx_a - mx) = 0
// or sum_b wy_b (dy_b - my) = 0, so A is diagonal and the least-squares fit of Eq. 9 is
// a_0 = sum W v / sum W, a_1 = sum W dx' v / sum W dx'^2, a_2 = sum W dy' v / sum W dy'^2.
// The interpolated value at the marker (dx = dy = 0) is a_0 - mx a_1 - my a_2 and the
// fitted gradient is (a_1, a_2): the same MLS solution as solving the 3x3 system, with
// the solve reduced to three reciprocals, done in double.
// ---------------------------------------------------------------------------------
constexpr double kMlsInvLen2 = 1.0 / (2.6 * 0.3 * 2.6 * 0.3);   // 1 / (r_w alpha)^2

template <typename C>
struct MlsW {
    int cx, cy;           // centre node (unwrapped)
    C wx[3], wy[3];       // axis weights, a or b = -1, 0, 1
    C dxp[3], dyp[3];     // centred offsets dx_a - mx, dy_b - my
    C k0, kx, ky;         // value weights: phi_ab = wx_a wy_b (k0 + kx dxp_a + ky dyp_b)
    C gx, gy;             // gradient weights: wx_a wy_b dxp_a gx, wx_a wy_b dyp_b gy
    C d0x, d0y;           // offset of the centre node from the point, (cx - X, cy - Y)
    bool ok;              // support inside the channel and the point sane
    bool sane;            // the point sane (else taken at the origin)
    // phi_k (Eq. 8) of support node (cx + a - 1, cy + b - 1)
    __device__ __forceinline__ C phi(int a, int b) const {
        return wx[a] * wy[b] * (k0 + kx * dxp[a] + ky * dyp[b]);
    }
};

// Whether the 3x3 support centred on node (cx, cy) stays inside the walls and, in an open
// channel, off the inlet and outlet columns.
__device__ __forceinline__ bool support_inside(const Lat& L, int cx, int cy) {
    return (!L.walls || (cy >= 1 && cy <= L.ny - 2)) && (!L.inflow || (cx >= 2 && cx <= L.nx - 3));
}

// Support geometry of a point: centre node and whether the 3x3 block stays inside the
// walls (and, in an open channel, off the open columns). A non-finite or runaway position (an unstable run) is moved to the origin so
// that every access stays inside the lattice, and reported as a support failure.
__device__ __forceinline__ bool support_centre(const Lat& L, double& X, double& Y, int& cx, int& cy,
                                               bool* sane_out = nullptr) {
    const bool sane = fabs(X) < 1e9 && fabs(Y) < 1e9;   // false for NaN too
    if (sane_out) *sane_out = sane;
    if (!sane) {
        X = 0.0;
        Y = 0.0;
    }
    cx = (int)floor(X + 0.5);
    cy = (int)floor(Y + 0.5);
    return sane && support_inside(L, cx, cy);
}

// Double reciprocal of a value known to lie well inside float range (the MLS weight
// sums and variances, between about 0.05 and 10): a float seed refined by two Newton
// steps r <- r (2 - x r), each of which doubles the number of correct bits (24 -> 48 ->
// full double precision).
__device__ __forceinline__ double rcp_bounded(double x) {
    double r = (double)__frcp_rn((float)x);
    r = r * (2.0 - x * r);
    r = r * (2.0 - x * r);
    return r;
}

// Shape functions of the point (X, Y). The offsets of the support from the point are
// formed in double (positions are double) and then held in the compute type; weights,
// sums, the solve (three reciprocals and the weighted means) and the application are in
// the compute type, the double solve's reciprocals refined from a float seed.
template <typename C>
__device__ __forceinline__ MlsW<C> mls_weights(int cx, int cy, C d0x, C d0y, bool ok);

template <typename C>
__device__ __forceinline__ MlsW<C> mls_setup(const Lat& L, double X, double Y) {
    int cx, cy;
    bool sane;
    const bool ok = support_centre(L, X, Y, cx, cy, &sane);
    MlsW<C> m = mls_weights<C>(cx, cy, C((double)cx - X), C((double)cy - Y), ok);   // offsets in [-1/2, 1/2]
    m.sane = sane;
    return m;
}

// A vertex's shape functions at X^n, kept from the kernel that computes them to the node
// update of the same step. Double: the whole MlsW (its solve is costly on the FP64 pipe).
// Single precision: only where the support lies, one aligned 16-byte record (centre node
// and offset; a NaN offset marks a position that was not sane), from which the update
// rebuilds the same weights in float: an array of 88-byte records would cost a
// scattered 32-byte sector per thread and word on every store and load.
struct __align__(16) MlsFrame {
    int cx, cy;
    float d0x, d0y;
};

template <typename C>
__device__ __forceinline__ void store_mls(void* base, long long g, const MlsW<C>& w) {
    if constexpr (sizeof(C) == 8) {
        reinterpret_cast<MlsW<C>*>(base)[g] = w;
    } else {
        reinterpret_cast<MlsFrame*>(base)[g] = MlsFrame{w.cx, w.cy, w.sane ? (float)w.d0x : __int_as_float(0x7fc00000),
                                                        (float)w.d0y};
    }
}

// The single-precision shape functions rebuilt from a stored frame.
template <typename C>
__device__ __forceinline__ MlsW<C> mls_from_frame(const Lat& L, const MlsFrame& f) {
    const bool sane = !isnan(f.d0x);
    const int cx = sane ? f.cx : 0, cy = sane ? f.cy : 0;
    MlsW<C> m = mls_weights<C>(cx, cy, sane ? C(f.d0x) : C(0), sane ? C(f.d0y) : C(0),
                               sane && support_inside(L, cx, cy));
    m.sane = sane;
    return m;
}

template <typename C>
__device__ __forceinline__ MlsW<C> load_mls(const Lat& L, const void* base, long long g) {
    if constexpr (sizeof(C) == 8) {
        return reinterpret_cast<const MlsW<C>*>(base)[g];
    } else {
        return mls_from_frame<C>(L, reinterpret_cast<const MlsFrame*>(base)[g]);
    }
}

// Single precision: shape functions of the point at the float offset (ox, oy) from a point
// whose own shape functions w are known (a probe beside a vertex). Its centre node and
// offset are found in float from w's centre node and offset, off the FP64 pipe; a
// non-finite or runaway offset (an unstable run) is taken as zero and reported.
template <typename C>
__device__ __forceinline__ MlsW<C> mls_near(const Lat& L, const MlsW<C>& w, float ox, float oy) {
    float px = ox - (float)w.d0x, py = oy - (float)w.d0y;   // from the centre node of w
    const bool sane = fabsf(px) < 1024.0f && fabsf(py) < 1024.0f;   // false for NaN too
    if (!sane) {
        px = 0.0f;
        py = 0.0f;
    }
    const float kx = floorf(px + 0.5f), ky = floorf(py + 0.5f);
    const int cx = w.cx + (int)kx, cy = w.cy + (int)ky;
    MlsW<C> m = mls_weights<C>(cx, cy, C(kx - px), C(ky - py), w.ok && sane && support_inside(L, cx, cy));
    m.sane = w.sane && sane;
    return m;
}

// Shape functions of the point whose centre node (cx, cy) lies at the offset (d0x, d0y)
// from it; `ok` from the support search.
template <typename C>
__device__ __forceinline__ MlsW<C> mls_weights(int cx, int cy, C d0x, C d0y, bool ok) {
    MlsW<C> m;
    m.cx = cx;
    m.cy = cy;
    m.d0x = d0x;
    m.d0y = d0y;
    m.ok = ok;
    m.sane = true;
    C dx[3], dy[3], sx0 = 0, sx1 = 0, sy0 = 0, sy1 = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        dx[a] = d0x + C(a - 1);
        dy[a] = d0y + C(a - 1);
        m.wx[a] = exp(-dx[a] * dx[a] * C(kMlsInvLen2));
        m.wy[a] = exp(-dy[a] * dy[a] * C(kMlsInvLen2));
        sx0 += m.wx[a];
        sx1 += m.wx[a] * dx[a];
        sy0 += m.wy[a];
        sy1 += m.wy[a] * dy[a];
    }
    if constexpr (sizeof(C) == 4) {
        // single precision: the solve in float as well (its error is of the order of the
        // float weighted sums it is applied to), off GB300's narrow FP64 pipe
        const C isx = C(1) / sx0, isy = C(1) / sy0;
        const C mx = sx1 * isx, my = sy1 * isy;
        C vx = 0, vy = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            m.dxp[a] = dx[a] - mx;
            m.dyp[a] = dy[a] - my;
            vx += m.wx[a] * m.dxp[a] * m.dxp[a];
            vy += m.wy[a] * m.dyp[a] * m.dyp[a];
        }
        const C rVx = (C(1) / vx) * isy, rVy = (C(1) / vy) * isx;
        m.k0 = isx * isy;
        m.kx = -mx * rVx;
        m.ky = -my * rVy;
        m.gx = rVx;
        m.gy = rVy;
        return m;
    }
    const double isx = rcp_bounded((double)sx0), isy = rcp_bounded((double)sy0);
    const double mx = (double)sx1 * isx, my = (double)sy1 * isy;
    C vx = 0, vy = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        m.dxp[a] = dx[a] - mx;
        m.dyp[a] = dy[a] - my;
        vx += m.wx[a] * m.dxp[a] * m.dxp[a];
        vy += m.wy[a] * m.dyp[a] * m.dyp[a];
    }
    const double rVx = rcp_bounded((double)vx) * isy;   // 1 / sum W dx'^2
    const double rVy = rcp_bounded((double)vy) * isx;   // 1 / sum W dy'^2
    m.k0 = C(isx * isy);
    m.kx = C(-mx * rVx);
    m.ky = C(-my * rVy);
    m.gx = C(rVx);
    m.gy = C(rVy);
    return m;
}

// Interpolated fluid quantities (Eq. 8) in the compute type.
template <typename C>
struct InterpT {
    C ux, uy, rho, p;
    C drho;   // rho - 1, kept apart so that single precision keeps its digits
    C dudx, dudy, dvdx, dvdy;
};
using Interp = InterpT<double>;

// Lattice moments at a node: density deviation and the Eq. 7 velocity (half of the
// uniform force plus the immersed-boundary force field).
template <typename C>
struct Mom {
    C drho, ux, uy;
};

template <typename S>
__device__ __forceinline__ Mom<typename St<S>::C> node_moments(const S* __restrict__ src, const Lat& L,
                                                               const double* __restrict__ fib, int x, int y) {
    using C = typename St<S>::C;
    C s[9];
    pull_all<S>(src, L, x, y, s);
    C drho, mx, my;
    moments<C>(s, drho, mx, my);
    const long long N = (long long)L.nx * L.ny;
    const long long n = (long long)y * L.nx + x;
    const C inv = C(1) / (C(1) + drho);
    Mom<C> m;
    m.drho = drho;
    const C gx = lat_c<C>(L.gx, L.gxf), gy = lat_c<C>(L.gy, L.gyf);   // C(g), rounded once on the host
    if (fib) {   // Eq. 7 with half of the uniform force and of the last spread force
        m.ux = (mx + C(0.5) * (gx + C(fib[n]))) * inv;
        m.uy = (my + C(0.5) * (gy + C(fib[N + n]))) * inv;
    } else {     // before any IB force (the Dynamic scheme's interpolations)
        m.ux = (mx + C(0.5) * gx) * inv;
        m.uy = (my + C(0.5) * gy) * inv;
    }
    return m;
}

// Lattice row of a support node (walls: clamped, the support is then flagged) and the
// periodic column.
__device__ __forceinline__ int support_row(const Lat& L, int yk) {
    if (L.walls) return yk < 0 ? 0 : (yk >= L.ny ? L.ny - 1 : yk);
    return wrapi(yk, L.ny);
}

// MLS interpolation (Eq. 8) from a moment source get(a, b) -> Mom for support node
// (cx + a - 1, cy + b - 1). Values in double, sums in the compute type.
template <typename C, bool GRAD, typename Get>
__device__ __forceinline__ void mls_apply(const MlsW<C>& m, Get&& get, InterpT<C>& o) {
    C r0 = 0, r1 = 0, r2 = 0, u0 = 0, u1 = 0, u2 = 0, v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
    for (int b = 0; b < 3; b++) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const Mom<C> q = get(a, b);
            const C w = m.wx[a] * m.wy[b];
            const C wx = w * m.dxp[a], wy = w * m.dyp[b];
            r0 += w * q.drho; r1 += wx * q.drho; r2 += wy * q.drho;
            u0 += w * q.ux; u1 += wx * q.ux; u2 += wy * q.ux;
            v0 += w * q.uy; v1 += wx * q.uy; v2 += wy * q.uy;
        }
    }
    o.ux = m.k0 * u0 + m.kx * u1 + m.ky * u2;
    o.uy = m.k0 * v0 + m.kx * v1 + m.ky * v2;
    o.drho = m.k0 * r0 + m.kx * r1 + m.ky * r2;
    o.rho = C(1) + o.drho;
    o.p = o.rho * C(1.0 / 3.0);
    if (GRAD) {
        o.dudx = m.gx * u1; o.dudy = m.gy * u2;
        o.dvdx = m.gx * v1; o.dvdy = m.gy * v2;
    }
}

// MLS interpolation of the fluid with given shape functions, straight from the
// populations (no tile).
template <typename S, bool GRAD>
__device__ bool mls_interp_with(const MlsW<typename St<S>::C>& m, const S* __restrict__ src, const Lat& L,
                                const double* __restrict__ fib, InterpT<typename St<S>::C>& o) {
    mls_apply<typename St<S>::C, GRAD>(m, [&](int a, int b) {
        return node_moments<S>(src, L, fib, wrapi(m.cx + a - 1, L.nx), support_row(L, m.cy + b - 1));
    }, o);
    return m.ok;
}

// MLS interpolation of the fluid at (X, Y) straight from the populations (no tile).
template <typename S, bool GRAD>
__device__ bool mls_interp(const S* __restrict__ src, const Lat& L, const double* __restrict__ fib, double X,
                           double Y, InterpT<typename St<S>::C>& o) {
    return mls_interp_with<S, GRAD>(mls_setup<typename St<S>::C>(L, X, Y), src, L, fib, o);
}

// Device status bits (sticky).
enum : unsigned {
    kStatUnstable = 1u,   // |u| > 0.3 or NaN in a collision
    kStatSupport = 2u,    // a support left the channel, or a position ran away
    kStatTimeout = 4u,    // a bounded wait gave up
    kStatList = 8u,       // touched-cell list full (entry dropped)
    kStatCell = 16u,      // a list entry outside the lattice (skipped)
    kStatRing = 32u,      // capsule parameters outside the launch's bounds (skipped)
    kStatGrid = 64u       // repulsion: a capsule outgrew the neighbour grid, or a bucket overflowed
};

// Small device block of counters and flags inside the arena.
struct DevCounters {
    int count[2];          // touched-cell list lengths (force buffers 0 and 1)
    unsigned status;       // sticky status bits
    int step_stamp;        // the patch's claim stamp (advanced by the last patch block to finish)
    int patch_blocks;      // patch blocks finished in the current launch
    int pad[3];
};

// Per-capsule parameters (device and host mirror).
struct CapsuleParams {
    int off, n;            // first vertex, vertex count
    double ks, kb, ka, m;  // Eq. 10, 12, 14 constants and per-vertex mass
    double A0, P0;         // stress-free area and perimeter
    int rigid;             // 1: a rigid particle (Section 2.3.1), state in Nodes::rb
};

}  // namespace lbmib
