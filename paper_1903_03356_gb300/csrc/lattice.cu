// Lattice kernels: fused pull collide-stream (Eq. 1-5), forced-node patch, start-up
// and read-back. Coclite et al., arXiv:1903.03356, Section 2.1-2.2.
//
// k_collide_stream is the HBM-bound hot loop. One warp owns a run of 32*V consecutive
// nodes of one row (V nodes per thread, 16 bytes of each population per thread). Every
// population is fetched with one aligned 16-byte load per thread; the +/-1 x shift of
// the pull is resolved with a warp shuffle of the neighbouring lane's edge element, and
// only the warp's edge lane issues one extra scalar load. Stores are aligned 16-byte
// stores of the node's own slots, so the kernel moves exactly 9 loads + 9 stores of
// the storage type per lattice update from HBM.
#include <algorithm>
#include <type_traits>

#include "lbmib_kernels.cuh"

namespace lbmib {

template <typename S>
struct Vec;
template <>
struct Vec<double> { static constexpr int V = 2; };
template <>
struct Vec<float> { static constexpr int V = 4; };
template <>
struct Vec<__half> { static constexpr int V = 4; };   // 8-byte vectors: keeps registers low

// Aligned vector load / store of V consecutive stored values (16 bytes for double and
// float, 8 bytes for half). Cache policy:
// load mode 0 = read-only path (ld.global.nc), 1 = streaming (ld.global.cs);
// store mode 0 = default write-back, 1 = streaming (st.global.cs, evict first).
template <int LM, typename T>
__device__ __forceinline__ T ldv(const T* p) {
    if constexpr (LM == 1) return __ldcs(p);
    else return __ldg(p);
}
template <int SM_, typename T>
__device__ __forceinline__ void stv(T* p, const T& v) {
    if constexpr (SM_ == 1) __stcs(p, v);
    else *p = v;
}

template <typename S, int LM>
__device__ __forceinline__ void ld_vec(const S* p, typename St<S>::C (&o)[Vec<S>::V], const Lat& L) {
    if constexpr (std::is_same<S, double>::value) {
        const double2 v = ldv<LM>(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    } else if constexpr (std::is_same<S, float>::value) {
        const float4 v = ldv<LM>(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const uint2 v = ldv<LM>(reinterpret_cast<const uint2*>(p));
        const __half2* h = reinterpret_cast<const __half2*>(&v);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float2 f = __half22float2(h[k]);
            o[2 * k] = f.x * L.inv_scale;
            o[2 * k + 1] = f.y * L.inv_scale;
        }
    }
}

template <typename S, int SMODE>
__device__ __forceinline__ void st_vec(S* p, const typename St<S>::C (&o)[Vec<S>::V], const Lat& L) {
    if constexpr (std::is_same<S, double>::value) {
        stv<SMODE>(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
    } else if constexpr (std::is_same<S, float>::value) {
        stv<SMODE>(reinterpret_cast<float4*>(p), make_float4(o[0], o[1], o[2], o[3]));
    } else {
        uint2 v;
        __half2* h = reinterpret_cast<__half2*>(&v);
#pragma unroll
        for (int k = 0; k < 2; k++) h[k] = __floats2half2_rn(o[2 * k] * L.scale, o[2 * k + 1] * L.scale);
        stv<SMODE>(reinterpret_cast<uint2*>(p), v);
    }
}

// Loads of population I for the V nodes x0 .. x0+V-1 of row y (pull of Eq. 1), split
// in two phases so that all nine populations' loads are in flight before any is used:
// issue() fetches the aligned 16-byte vector of the source row (at a wall, of the node's
// own opposite population) and, for an edge lane, the one scalar that no neighbouring
// lane holds; resolve() shifts by -e_x through warp shuffles. All 32 lanes of the warp
// call both with the same y. A lane whose chunk crosses the end of the row ("ragged",
// only when nx is not a multiple of V) keeps its raw vector for its neighbours'
// shuffles and gathers its own shifted values element-wise in resolve().
template <typename S, int I, int LM>
struct PopLoad {
    using C = typename St<S>::C;
    static constexpr int V = Vec<S>::V;
    C v[V];
    C edge;

    __device__ __forceinline__ bool at_wall(const Lat& L, int y) const {
        constexpr int EY = ey(I);
        return EY != 0 && L.walls && (y - EY < 0 || y - EY >= L.ny);
    }
    __device__ __forceinline__ const S* row_ptr(const S* __restrict__ src, const Lat& L, int y) const {
        constexpr int EY = ey(I);
        if (at_wall(L, y)) return src + (long long)opp(I) * L.plane + (long long)y * L.pitch;
        const int ys = EY != 0 ? wrapi(y - EY, L.ny) : y;
        return src + (long long)I * L.plane + (long long)ys * L.pitch;
    }
    __device__ __forceinline__ void issue(const S* __restrict__ src, const Lat& L, int x0, int y, int lane,
                                          bool active) {
        constexpr int EX = ex(I);
        const S* row = row_ptr(src, L, y);
        edge = C(0);
        if (active) {
            // x0 < nx <= pitch and both are multiples of V: the vector stays inside the row
            ld_vec<S, LM>(row + x0, v, L);
        } else {
#pragma unroll
            for (int j = 0; j < V; j++) v[j] = C(0);
        }
        if (!at_wall(L, y) && active) {
            if (EX == 1 && lane == 0) edge = St<S>::ld(row + wrapi(x0 - 1, L.nx), L);
            // the next lane's chunk is missing or ragged: fetch x0 + V directly
            if (EX == -1 && (lane == 31 || x0 + 2 * V > L.nx)) edge = St<S>::ld(row + wrapi(x0 + V, L.nx), L);
        }
    }
    __device__ __forceinline__ void resolve(const S* __restrict__ src, const Lat& L, int x0, int y, int lane,
                                            bool active, bool full, C (&out)[V]) const {
        constexpr int EX = ex(I);
        if (at_wall(L, y)) {  // warp-uniform
            constexpr int J = opp(I);
            const C uw = y - ey(I) < 0 ? lat_c<C>(L.ub, L.ubf) : lat_c<C>(L.ut, L.utf);
            const C corr = C(6) * wgt<C>(J) * C(ex(J)) * uw;
#pragma unroll
            for (int j = 0; j < V; j++) out[j] = v[j] - corr;
        } else if (EX == 0) {
#pragma unroll
            for (int j = 0; j < V; j++) out[j] = v[j];
        } else if (EX == 1) {  // value at x - 1
            C prev = __shfl_up_sync(0xffffffffu, v[V - 1], 1);
            if (lane == 0) prev = edge;
            out[0] = prev;
#pragma unroll
            for (int j = 1; j < V; j++) out[j] = v[j - 1];
        } else {               // value at x + 1
            C next = __shfl_down_sync(0xffffffffu, v[0], 1);
            if (lane == 31 || x0 + 2 * V > L.nx) next = edge;
#pragma unroll
            for (int j = 0; j < V - 1; j++) out[j] = v[j + 1];
            out[V - 1] = next;
        }
        if (active && !full) {  // ragged chunk: element-wise, with the pull's wrap
            const S* row = row_ptr(src, L, y);
            const bool wall = at_wall(L, y);
            const C uw = y - ey(I) < 0 ? lat_c<C>(L.ub, L.ubf) : lat_c<C>(L.ut, L.utf);
            const C corr = wall ? C(6) * wgt<C>(opp(I)) * C(ex(opp(I))) * uw : C(0);
#pragma unroll
            for (int j = 0; j < V; j++) {
                const int x = x0 + j;
                out[j] = x < L.nx ? (wall ? St<S>::ld(row + x, L) - corr : St<S>::ld(row + wrapi(x - EX, L.nx), L))
                                  : C(0);
            }
        }
    }
};

template <typename S, int LM, int SMODE, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_collide_stream(const S* __restrict__ src, S* __restrict__ dst,
                                                             Lat L, unsigned* __restrict__ status) {
    using C = typename St<S>::C;
    constexpr int V = Vec<S>::V;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * BS + threadIdx.x) >> 5;
    const int segs = (L.nx + 32 * V - 1) / (32 * V);
    if (gw >= (long long)segs * L.ny) return;  // whole warps only
    const int y = (int)(gw / segs);
    const int seg = (int)(gw - (long long)y * segs);
    const int x0 = (seg * 32 + lane) * V;
    const bool active = x0 < L.nx;
    const bool full = x0 + V <= L.nx;

    PopLoad<S, 0, LM> p0; PopLoad<S, 1, LM> p1; PopLoad<S, 2, LM> p2;
    PopLoad<S, 3, LM> p3; PopLoad<S, 4, LM> p4; PopLoad<S, 5, LM> p5;
    PopLoad<S, 6, LM> p6; PopLoad<S, 7, LM> p7; PopLoad<S, 8, LM> p8;
    p0.issue(src, L, x0, y, lane, active); p1.issue(src, L, x0, y, lane, active);
    p2.issue(src, L, x0, y, lane, active); p3.issue(src, L, x0, y, lane, active);
    p4.issue(src, L, x0, y, lane, active); p5.issue(src, L, x0, y, lane, active);
    p6.issue(src, L, x0, y, lane, active); p7.issue(src, L, x0, y, lane, active);
    p8.issue(src, L, x0, y, lane, active);
    C f[9][V];
    p0.resolve(src, L, x0, y, lane, active, full, f[0]); p1.resolve(src, L, x0, y, lane, active, full, f[1]);
    p2.resolve(src, L, x0, y, lane, active, full, f[2]); p3.resolve(src, L, x0, y, lane, active, full, f[3]);
    p4.resolve(src, L, x0, y, lane, active, full, f[4]); p5.resolve(src, L, x0, y, lane, active, full, f[5]);
    p6.resolve(src, L, x0, y, lane, active, full, f[6]); p7.resolve(src, L, x0, y, lane, active, full, f[7]);
    p8.resolve(src, L, x0, y, lane, active, full, f[8]);

    const C gx = lat_c<C>(L.gx, L.gxf), gy = lat_c<C>(L.gy, L.gyf), om = lat_c<C>(L.omega, L.omegaf);
    bool bad = false;
    if constexpr (std::is_same<S, __half>::value) {
        // FP16 storage (issue-bound): nodes in pairs, two lanes per instruction, as in the
        // packed FP16 kernel, whose results this kernel reproduces bit for bit
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            F2 s[9];
#pragma unroll
            for (int i = 0; i < 9; i++) s[i] = F2{f[i][j], f[i][j + 1]};
            const F2 usq = collide2(s, gx, gy, om);
            bad |= !(usq.x < 0.09f) || !(usq.y < 0.09f);  // |u| > 0.3 or NaN
#pragma unroll
            for (int i = 0; i < 9; i++) {
                f[i][j] = s[i].x;
                f[i][j + 1] = s[i].y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; j++) {
            C s[9];
#pragma unroll
            for (int i = 0; i < 9; i++) s[i] = f[i][j];
            const C usq = collide<C>(s, gx, gy, om);
            bad |= !(usq < C(0.09));  // |u| > 0.3 or NaN
#pragma unroll
            for (int i = 0; i < 9; i++) f[i][j] = s[i];
        }
    }
    if (full) {
#pragma unroll
        for (int i = 0; i < 9; i++)
            st_vec<S, SMODE>(dst + (long long)i * L.plane + (long long)y * L.pitch + x0, f[i], L);
    } else if (active) {
#pragma unroll
        for (int i = 0; i < 9; i++)
#pragma unroll
            for (int j = 0; j < V; j++)
                if (x0 + j < L.nx) St<S>::st(dst + (long long)i * L.plane + (long long)y * L.pitch + x0 + j, f[i][j], L);
    }
    if (__any_sync(0xffffffffu, bad && active) && lane == 0) atomicOr(status, kStatUnstable);
}

// FP16 storage: one warp owns 256 consecutive nodes of a row, 8 per thread, each
// population fetched with one aligned 16-byte load and kept packed (four half2
// registers) until its node pair is collided; the results are packed back and stored
// as 16-byte vectors. This keeps the bytes in flight per thread at the FP32 kernel's
// (9 x 16 B) without holding 72 floats in registers. The kernel is bound to 6 blocks of
// 128 per SM (80 registers, a few spilled values): the chains of packed instructions
// need the warps more than the spilled registers cost (4, 5, 6, 7, 8 blocks: 119, 130,
// 136, 132, 127 GLUPS on a 16384 x 8192 lattice; 8-byte half stores instead of the
// 16-byte ones, to spill less, 129).
template <int I>
struct PopH {
    __half2 h[4];   // halves of the source row at x0 .. x0+7 (own opposite row at a wall)
    __half edge;    // the element no neighbouring lane holds

    __device__ __forceinline__ bool at_wall(const Lat& L, int y) const {
        constexpr int EY = ey(I);
        return EY != 0 && L.walls && (y - EY < 0 || y - EY >= L.ny);
    }
    __device__ __forceinline__ const __half* row_ptr(const __half* __restrict__ src, const Lat& L, int y) const {
        constexpr int EY = ey(I);
        if (at_wall(L, y)) return src + (long long)opp(I) * L.plane + (long long)y * L.pitch;
        const int ys = EY != 0 ? wrapi(y - EY, L.ny) : y;
        return src + (long long)I * L.plane + (long long)ys * L.pitch;
    }
    __device__ __forceinline__ void issue(const __half* __restrict__ src, const Lat& L, int x0, int y, int lane,
                                          bool active) {
        constexpr int EX = ex(I);
        const __half* row = row_ptr(src, L, y);
        edge = __float2half(0.0f);
        uint4 raw = make_uint4(0u, 0u, 0u, 0u);
        // x0 < nx <= pitch, both multiples of 8: the vector stays inside the padded row
        if (active) raw = __ldg(reinterpret_cast<const uint4*>(row + x0));
        const __half2* hp = reinterpret_cast<const __half2*>(&raw);
#pragma unroll
        for (int k = 0; k < 4; k++) h[k] = hp[k];
        if (!at_wall(L, y) && active) {
            if (EX == 1 && lane == 0) edge = __ldg(row + wrapi(x0 - 1, L.nx));
            if (EX == -1 && (lane == 31 || x0 + 16 > L.nx)) edge = __ldg(row + wrapi(x0 + 8, L.nx));
        }
    }
    __device__ __forceinline__ __half elem(int j) const { return (j & 1) ? __high2half(h[j >> 1]) : __low2half(h[j >> 1]); }
    // the neighbouring element across the lane boundary (all 32 lanes call this together)
    __device__ __forceinline__ __half across(const Lat& L, int x0, int lane) const {
        constexpr int EX = ex(I);
        if (EX == 1) {
            const __half p = __shfl_up_sync(0xffffffffu, elem(7), 1);
            return lane == 0 ? edge : p;
        }
        const __half nx = __shfl_down_sync(0xffffffffu, elem(0), 1);
        return (lane == 31 || x0 + 16 > L.nx) ? edge : nx;
    }
};

template <int I>
__device__ __forceinline__ float pop_value(const PopH<I>& p, __half across, int j, bool wall, float corr,
                                           float inv_scale) {
    constexpr int EX = ex(I);
    __half v;
    if (wall || EX == 0) v = p.elem(j);
    else if (EX == 1) v = j == 0 ? across : p.elem(j - 1);
    else v = j == 7 ? across : p.elem(j + 1);
    // unscaling never fused with the wall correction (as St<__half>::ld)
    return __fmul_rn(__half2float(v), inv_scale) - (wall ? corr : 0.0f);
}

// The ragged chunk at the end of a row of the packed FP16 kernel (nx not a multiple of
// 8): element-wise loads with the pull's own wrap, nodes in pairs with the lane arithmetic
// of the full chunks (a missing partner repeats the node and is not stored). Run
// by k_ragged_h. Returns whether a node is unstable.
__device__ __forceinline__ bool ragged_chunk_h(const __half* __restrict__ src, __half* __restrict__ dst, const Lat& L,
                                            int x0, int y, float gx, float gy, float om) {
    bool bad = false;
    for (int j = 0; j < 8 && x0 + j < L.nx; j += 2) {
        const bool two = x0 + j + 1 < L.nx;
        float a[9], b[9];
        pull_all<__half>(src, L, x0 + j, y, a);
        pull_all<__half>(src, L, two ? x0 + j + 1 : x0 + j, y, b);
        F2 s[9];
#pragma unroll
        for (int i = 0; i < 9; i++) s[i] = F2{a[i], b[i]};
        const F2 usq = collide2(s, gx, gy, om);
        bad |= !(usq.x < 0.09f) || (two && !(usq.y < 0.09f));
#pragma unroll
        for (int i = 0; i < 9; i++) {
            St<__half>::st(dst + (long long)i * L.plane + (long long)y * L.pitch + x0 + j, s[i].x, L);
            if (two) St<__half>::st(dst + (long long)i * L.plane + (long long)y * L.pitch + x0 + j + 1, s[i].y, L);
        }
    }
    return bad;
}

template <int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_collide_stream_h(const __half* __restrict__ src,
                                                               __half* __restrict__ dst, Lat L,
                                                               unsigned* __restrict__ status) {
    constexpr int V = 8;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * BS + threadIdx.x) >> 5;
    const int segs = (L.nx + 32 * V - 1) / (32 * V);
    if (gw >= (long long)segs * L.ny) return;   // whole warps only
    const int y = (int)(gw / segs);
    const int seg = (int)(gw - (long long)y * segs);
    const int x0 = (seg * 32 + lane) * V;
    const bool active = x0 < L.nx;
    const bool full = x0 + V <= L.nx;

    PopH<0> p0; PopH<1> p1; PopH<2> p2; PopH<3> p3; PopH<4> p4;
    PopH<5> p5; PopH<6> p6; PopH<7> p7; PopH<8> p8;
    p0.issue(src, L, x0, y, lane, active); p1.issue(src, L, x0, y, lane, active);
    p2.issue(src, L, x0, y, lane, active); p3.issue(src, L, x0, y, lane, active);
    p4.issue(src, L, x0, y, lane, active); p5.issue(src, L, x0, y, lane, active);
    p6.issue(src, L, x0, y, lane, active); p7.issue(src, L, x0, y, lane, active);
    p8.issue(src, L, x0, y, lane, active);
    const __half a1 = p1.across(L, x0, lane), a3 = p3.across(L, x0, lane), a5 = p5.across(L, x0, lane);
    const __half a6 = p6.across(L, x0, lane), a7 = p7.across(L, x0, lane), a8 = p8.across(L, x0, lane);
    // wall corrections -6 w_j (e_j . u_w) of the reflected populations (Section 2.1, R2)
    const bool lo = L.walls && y == 0, hi = L.walls && y == L.ny - 1;
    const float cw = 6.0f / 36.0f;
    const float c2 = 0.0f;   // populations 2 and 4 reflect populations without an x component
    const float c5 = -cw * L.ubf, c6 = cw * L.ubf;   // bottom wall: 5 <- 7 (e_x -1), 6 <- 8 (e_x +1)
    const float c7 = cw * L.utf, c8 = -cw * L.utf;   // top wall: 7 <- 5 (e_x +1), 8 <- 6 (e_x -1)
    const float gx = L.gxf, gy = L.gyf, om = L.omegaf, is = L.inv_scale, sc = L.scale;
    uint4 out[9];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        // nodes 2q and 2q + 1, two lanes per instruction
        F2 s[9];
#pragma unroll
        for (int t = 0; t < 2; t++) {
            const int j = 2 * q + t;
            float* lane = t == 0 ? &s[0].x : &s[0].y;   // lane t of every population pair
            lane[0 * 2] = pop_value(p0, a1, j, false, 0.0f, is);
            lane[1 * 2] = pop_value(p1, a1, j, false, 0.0f, is);
            lane[2 * 2] = pop_value(p2, a1, j, lo, c2, is);
            lane[3 * 2] = pop_value(p3, a3, j, false, 0.0f, is);
            lane[4 * 2] = pop_value(p4, a1, j, hi, c2, is);
            lane[5 * 2] = pop_value(p5, a5, j, lo, c5, is);
            lane[6 * 2] = pop_value(p6, a6, j, lo, c6, is);
            lane[7 * 2] = pop_value(p7, a7, j, hi, c7, is);
            lane[8 * 2] = pop_value(p8, a8, j, hi, c8, is);
        }
        const F2 usq = collide2(s, gx, gy, om);
        bad |= !(usq.x < 0.09f) || !(usq.y < 0.09f);
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const F2 v = s[i] * f2(sc);
            const __half2 hv = __floats2half2_rn(v.x, v.y);
            (&out[i].x)[q] = *reinterpret_cast<const unsigned*>(&hv);
        }
    }
    if (full) {
#pragma unroll
        for (int i = 0; i < 9; i++)
            *reinterpret_cast<uint4*>(dst + (long long)i * L.plane + (long long)y * L.pitch + x0) = out[i];
    }   // a ragged chunk at the end of a row is k_ragged_h's
    if (__any_sync(0xffffffffu, bad && full) && lane == 0) atomicOr(status, kStatUnstable);
}

// The ragged chunk at the end of every row of the packed FP16 kernel (nx not a multiple
// of 8), one thread per row, launched after it: a separate kernel keeps the element-wise
// path out of the hot kernel's registers.
__global__ void __launch_bounds__(128) k_ragged_h(const __half* __restrict__ src, __half* __restrict__ dst, Lat L,
                                                  unsigned* __restrict__ status) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= L.ny) return;
    if (ragged_chunk_h(src, dst, L, L.nx / 8 * 8, y, L.gxf, L.gyf, L.omegaf)) atomicOr(status, kStatUnstable);
}

// Forced-node patch: the nodes of the current touched-cell list collide with the total
// force g + f_ib (Eq. 4-5) instead of g. The lattice update has just written their
// unforced post-collision populations in place, and those determine the forced ones
// (force_node: the mass and momentum of the unforced collision give rho and u), so the
// patch reads and writes each node's own nine slots and nothing else of the lattice. A
// node that several capsules' tiles cover is listed more than once: the first thread to
// claim it (an atomic exchange of this launch's stamp, issued with the loads) patches it,
// the others leave it. The last block to finish advances the stamp. Also clears the
// previous force buffer at the previous list (its last reader has run).
template <typename S>
__global__ void __launch_bounds__(256) k_patch(S* __restrict__ dst, Lat L, const double* __restrict__ fib_c,
                                               const int* __restrict__ list_c, double* __restrict__ fib_p,
                                               const int* __restrict__ list_p, int* __restrict__ mark,
                                               DevCounters* ctr, int c, int capacity) {
    using C = typename St<S>::C;
    const long long N = (long long)L.nx * L.ny;
    int nc = ctr->count[c];
    int np = ctr->count[1 - c];
    const int stamp = ctr->step_stamp + 1;
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (nc > capacity || np > capacity) {
        if (t0 == 0) atomicOr(&ctr->status, kStatList);
        nc = nc > capacity ? capacity : nc;
        np = np > capacity ? capacity : np;
    }
    const C gx = lat_c<C>(L.gx, L.gxf), gy = lat_c<C>(L.gy, L.gyf), om = lat_c<C>(L.omega, L.omegaf);
    // two list entries per thread and pass, all their loads and claims issued before
    // either is used (the kernel waits on memory latency, not bandwidth)
    for (int k = t0; k < nc; k += 2 * stride) {
        int cell[2] = {list_c[k], k + stride < nc ? list_c[k + stride] : -1};
        bool use[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            use[q] = cell[q] >= 0 && (long long)cell[q] < N;
            if (!use[q] && (q == 0 || k + stride < nc)) atomicOr(&ctr->status, kStatCell);
            if (!use[q]) cell[q] = 0;
        }
        long long at[2];
        C s[2][9];
        double fx[2], fy[2];
        int old[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int y = cell[q] / L.nx;
            at[q] = (long long)y * L.pitch + (cell[q] - y * L.nx);
            old[q] = use[q] ? atomicExch(mark + cell[q], stamp) : stamp;
#pragma unroll
            for (int i = 0; i < 9; i++) s[q][i] = St<S>::ld(dst + (long long)i * L.plane + at[q], L);
            fx[q] = fib_c[cell[q]];
            fy[q] = fib_c[N + cell[q]];
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
            if (!use[q] || old[q] == stamp) continue;   // not a cell, or claimed by another entry
            const C usq = force_node<C>(s[q], gx, gy, C(L.gx + fx[q]), C(L.gy + fy[q]), om);
            if (!(usq < C(0.09))) atomicOr(&ctr->status, kStatUnstable);
#pragma unroll
            for (int i = 0; i < 9; i++) St<S>::st(dst + (long long)i * L.plane + at[q], s[q][i], L);
        }
    }
    for (int k = t0; k < np; k += stride) {
        const int cell = list_p[k];
        if (cell < 0 || (long long)cell >= N) {
            atomicOr(&ctr->status, kStatCell);
            continue;
        }
        fib_p[cell] = 0.0;
        fib_p[N + cell] = 0.0;
    }
    // the stamp stays fixed until every block has read it: the last block advances it
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctr->patch_blocks, 1) == (int)gridDim.x - 1) {
            ctr->patch_blocks = 0;
            ctr->step_stamp = stamp;
        }
    }
}

// Start-up: post-collision populations whose pull gives the Eq. 2 equilibrium of the
// fields (rho, ux, uy) at every node ("un-streaming" through walls and periodic edges).
template <typename S>
__global__ void k_init(S* __restrict__ dst, Lat L, const double* __restrict__ rho,
                       const double* __restrict__ ux, const double* __restrict__ uy) {
    using C = typename St<S>::C;
    const long long N = (long long)L.nx * L.ny;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int y = (int)(n / L.nx), x = (int)(n - (long long)y * L.nx);
    if constexpr (sizeof(C) == 4) {
        // single precision: each node converts its own fields once (rho - 1 formed in
        // double) and pushes its nine shifted equilibria to the nodes that pull them,
        // which keeps the start-up off the narrow FP64 pipe; a population that would be
        // pulled from beyond a wall is this node's own reflected one
        const double r = rho ? rho[n] : 1.0;
        const C dr = C(r - 1.0), rr = C(r), u = ux ? C(ux[n]) : C(0), v = uy ? C(uy[n]) : C(0);
        const C u15 = C(1.5) * (u * u + v * v);
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const C eu = C(ex(i)) * u + C(ey(i)) * v;
            const C w = wgt<C>(i);
            const int ys = y - ey(i);
            if (!L.walls || (ys >= 0 && ys < L.ny)) {
                const int xs = wrapi(x - ex(i), L.nx), yw = L.walls ? ys : wrapi(ys, L.ny);
                St<S>::st(dst + (long long)i * L.plane + (long long)yw * L.pitch + xs,
                          w * (dr + rr * (C(3) * eu + C(4.5) * eu * eu - u15)), L);
            }
            const int yt = y + ey(i);
            if (L.walls && (yt < 0 || yt >= L.ny)) {
                // f_opp(i) of this node's own fields (e_opp(i) . u = -e_i . u), with the
                // moving-wall correction
                const C corr = C(6.0 * wgt<double>(i) * ex(i) * (yt < 0 ? L.ub : L.ut));
                St<S>::st(dst + (long long)i * L.plane + (long long)y * L.pitch + x,
                          w * (dr + rr * (C(-3) * eu + C(4.5) * eu * eu - u15)) + corr, L);
            }
        }
    } else {
    #pragma unroll
        for (int i = 0; i < 9; i++) {
            int xt = x + ex(i), yt = y + ey(i);
            int k = i;
            double corr = 0.0;
            if (L.walls && (yt < 0 || yt >= L.ny)) {
                // consumed by this node as the reflected population opp(i)
                k = opp(i);
                corr = 6.0 * wgt<double>(i) * ex(i) * (yt < 0 ? L.ub : L.ut);
                xt = x;
                yt = y;
            } else {
                xt = wrapi(xt, L.nx);
                yt = wrapi(yt, L.ny);
            }
            const long long m = (long long)yt * L.nx + xt;
            const double r = rho ? rho[m] : 1.0, u = ux ? ux[m] : 0.0, v = uy ? uy[m] : 0.0;
            const double eu = ex(k) * u + ey(k) * v;
            const double feq = wgt<double>(k) * r * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * (u * u + v * v));
            St<S>::st(dst + (long long)i * L.plane + (long long)y * L.pitch + x, C(feq - wgt<double>(i) + corr), L);
        }
    }
}

// Read-back: rho (Eq. 6) and u (Eq. 7, half of g + f_ib) at every node, in double.
template <typename S>
__global__ void k_macros(const S* __restrict__ src, Lat L, OpenBC ob, const double* __restrict__ fib,
                         double* __restrict__ rho, double* __restrict__ ux, double* __restrict__ uy) {
    using C = typename St<S>::C;
    const long long N = (long long)L.nx * L.ny;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int y = (int)(n / L.nx), x = (int)(n - (long long)y * L.nx);
    C s[9];
    pull_all<S>(src, L, x, y, s, &ob);
    C drho, mx, my;
    moments<C>(s, drho, mx, my);
    rho[n] = 1.0 + (double)drho;
    if constexpr (sizeof(C) == 4) {   // single precision: the velocity in float, off the FP64 pipe
        const C inv = C(1) / (C(1) + drho);
        ux[n] = (double)((mx + C(0.5) * (C(L.gx) + C(fib[n]))) * inv);
        uy[n] = (double)((my + C(0.5) * (C(L.gy) + C(fib[N + n]))) * inv);
    } else {
        const double r = 1.0 + (double)drho;
        ux[n] = ((double)mx + 0.5 * (L.gx + fib[n])) / r;
        uy[n] = ((double)my + 0.5 * (L.gy + fib[N + n])) / r;
    }
}

// Read-back: unshifted pre-collision populations i0 .. i0+2 in double.
template <typename S>
__global__ void k_populations(const S* __restrict__ src, Lat L, OpenBC ob, int i0, double* __restrict__ out) {
    const long long N = (long long)L.nx * L.ny;
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int y = (int)(n / L.nx), x = (int)(n - (long long)y * L.nx);
    typename St<S>::C s[9];
    pull_all<S>(src, L, x, y, s, &ob);
    for (int k = 0; k < 3 && i0 + k < 9; k++) {
        const int i = i0 + k;
        double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        out[k * N + n] = (double)s[i] + w;
    }
}

// Open channel: redo the update of the inlet and outlet columns (2 ny nodes), whose
// pulls across x = 0 and x = nx - 1 the lattice kernel took through the periodic wrap:
// pull_all applies the Zou-He closure there, then the node collides with the uniform
// force (Eq. 4-5) like every other node. Runs after the lattice kernel, on its output.
template <typename S>
__global__ void __launch_bounds__(128) k_open_columns(const S* __restrict__ src, S* __restrict__ dst, Lat L,
                                                      OpenBC ob, unsigned* status) {
    using C = typename St<S>::C;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * L.ny) return;
    const int y = k >> 1, x = (k & 1) ? L.nx - 1 : 0;
    C s[9];
    pull_all<S>(src, L, x, y, s, &ob);
    const C usq = collide<C>(s, lat_c<C>(L.gx, L.gxf), lat_c<C>(L.gy, L.gyf), lat_c<C>(L.omega, L.omegaf));
    if (!(usq < C(0.09))) atomicOr(status, kStatUnstable);
#pragma unroll
    for (int i = 0; i < 9; i++) St<S>::st(dst + (long long)i * L.plane + (long long)y * L.pitch + x, s[i], L);
}

// ---------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// variant: bits 0-11 block size (128 or 256; default 256); bit 18 asks for four resident
// blocks per SM (register cap 64 at 256 threads) instead of three.
template <typename S>
void launch_collide_stream(const void* src, void* dst, const Lat& L, unsigned* status, int variant,
                           cudaStream_t s) {
    constexpr int V = Vec<S>::V;
    const int bs = (variant & 0xfff) == 128 ? 128 : 256;
    const bool occ4 = (variant >> 18) & 1;
    const long long segs = (L.nx + 32 * V - 1) / (32 * V);
    const long long threads = segs * L.ny * 32;
    const unsigned g = blocks_for(threads, bs);
    const S* a = (const S*)src;
    S* b = (S*)dst;
    if constexpr (std::is_same<S, __half>::value) {
        if (variant & (1 << 19)) {   // packed 16-byte FP16 kernel, 8 nodes per thread
            const long long segs8 = (L.nx + 255) / 256;
            const unsigned g8 = blocks_for(segs8 * L.ny * 32, bs);
            if (bs == 128) k_collide_stream_h<128, 6><<<g8, 128, 0, s>>>(a, b, L, status);
            else k_collide_stream_h<256, 3><<<g8, 256, 0, s>>>(a, b, L, status);
            if (L.nx % 8) k_ragged_h<<<blocks_for(L.ny, 128), 128, 0, s>>>(a, b, L, status);
            return;
        }
    }
    if (bs == 256 && !occ4) k_collide_stream<S, 0, 0, 256, 3><<<g, 256, 0, s>>>(a, b, L, status);
    else if (bs == 256) k_collide_stream<S, 0, 0, 256, 4><<<g, 256, 0, s>>>(a, b, L, status);
    else if (!occ4) k_collide_stream<S, 0, 0, 128, 6><<<g, 128, 0, s>>>(a, b, L, status);
    else k_collide_stream<S, 0, 0, 128, 8><<<g, 128, 0, s>>>(a, b, L, status);
}

template <typename S>
void launch_patch(void* dst, const Lat& L, const double* fib_c, const int* list_c, double* fib_p,
                  const int* list_p, int* mark, DevCounters* ctr, int c, int capacity, long long vertices,
                  cudaStream_t s) {
    // a grid-stride loop over the touched list, whose length only the device knows, two
    // entries per thread and pass, sized for 1.1 entries per vertex (the 16384 x 8192
    // benchmark lists 2.2e6 nodes for 2.1e6 vertices: one pass, and no idle blocks; a
    // longer list takes more passes), at most 6144 blocks of 256
    const long long want = (11 * (vertices > 0 ? vertices : 1) + 9) / 10;
    int grid = (int)blocks_for((std::min<long long>(want, capacity > 0 ? capacity : 1) + 1) / 2, 256);
    if (grid > 6144) grid = 6144;
    k_patch<S><<<grid, 256, 0, s>>>((S*)dst, L, fib_c, list_c, fib_p, list_p, mark, ctr, c, capacity);
}

template <typename S>
void launch_open_columns(const void* src, void* dst, const Lat& L, const OpenBC& ob, unsigned* status,
                         cudaStream_t s) {
    k_open_columns<S><<<blocks_for(2LL * L.ny, 128), 128, 0, s>>>((const S*)src, (S*)dst, L, ob, status);
}

template <typename S>
void launch_init(void* dst, const Lat& L, const double* rho, const double* ux, const double* uy, cudaStream_t s) {
    k_init<S><<<blocks_for((long long)L.nx * L.ny, 256), 256, 0, s>>>((S*)dst, L, rho, ux, uy);
}

template <typename S>
void launch_macros(const void* src, const Lat& L, const OpenBC& ob, const double* fib, double* rho, double* ux,
                   double* uy, cudaStream_t s) {
    k_macros<S><<<blocks_for((long long)L.nx * L.ny, 256), 256, 0, s>>>((const S*)src, L, ob, fib, rho, ux, uy);
}

template <typename S>
void launch_populations(const void* src, const Lat& L, const OpenBC& ob, int i0, double* out, cudaStream_t s) {
    k_populations<S><<<blocks_for((long long)L.nx * L.ny, 256), 256, 0, s>>>((const S*)src, L, ob, i0, out);
}

#define LBMIB_INSTANTIATE_LATTICE(S)                                                                  \
    template void launch_collide_stream<S>(const void*, void*, const Lat&, unsigned*, int, cudaStream_t); \
    template void launch_patch<S>(void*, const Lat&, const double*, const int*, double*, const int*,   \
                                  int*, DevCounters*, int, int, long long, cudaStream_t);             \
    template void launch_open_columns<S>(const void*, void*, const Lat&, const OpenBC&, unsigned*,     \
                                         cudaStream_t);                                               \
    template void launch_init<S>(void*, const Lat&, const double*, const double*, const double*,      \
                                 cudaStream_t);                                                       \
    template void launch_macros<S>(const void*, const Lat&, const OpenBC&, const double*, double*,     \
                                   double*, double*, cudaStream_t);                                   \
    template void launch_populations<S>(const void*, const Lat&, const OpenBC&, int, double*, cudaStream_t);

LBMIB_INSTANTIATE_LATTICE(double)
LBMIB_INSTANTIATE_LATTICE(float)
LBMIB_INSTANTIATE_LATTICE(__half)

}  // namespace lbmib
