// Batched persistent launch: many independent capsule cases (each its own small
// lattice and capsule) advanced by one kernel launch with the Kinematic scheme
// (Section 2.4, steps i-viii; Eq. 1-14 and 25).
//
// One CTA owns one case for all the steps of a launch: it takes the next case from an
// atomic queue (cases ordered largest first), keeps the capsule ring in shared memory
// across steps, and per step
//   1. computes the internal forces (Eq. 11, 13, 14) and spreads them into a shared
//      force tile over the ring's bounding box (step iii);
//   2. sweeps the case's lattice: pull, BGK + Guo collision with g plus the tile force
//      where the node lies in the tile (Eq. 4-5), store — so no global force field and no
//      separate patch are needed;
//   3. fills a shared moment tile from the new populations and advances the ring with
//      the interpolated velocity (Eq. 8, Eq. 25).
// No CTA ever waits for another (cases are independent), so the launch has no grid-wide
// barrier. A launch is replayed from a captured CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbmib.h"
#include "ring.cuh"

namespace lbmib {

struct BatchCase {
    Lat L;
    long long pops;       // element offset of buffer 0 in the population pool (buffer 1 at +9 plane)
    int cur;              // buffer holding the latest post-collision populations
    int off, n;           // vertex range (n = 0: no capsule)
    int age;              // steps taken by the capsule
};

struct BatchDev {
    void* pops;
    BatchCase* cases;
    const int* order;     // processing order (largest lattice first)
    int* queue;           // next entry of `order` to take
    unsigned* status;
    Nodes nd;             // vertex arrays of all cases; caps holds each case's membrane constants
    int ncases;
};

// Two adjacent stored values (x, x + 1; x even, so the pair is aligned) as the compute
// type. Plain loads and stores: the CTA rewrites its case's populations every step.
template <typename S>
__device__ __forceinline__ void ld_pair(const S* p, const Lat& L, typename St<S>::C& a, typename St<S>::C& b) {
    if constexpr (sizeof(S) == 8) {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x;
        b = v.y;
    } else if constexpr (sizeof(S) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x;
        b = v.y;
    } else {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
        a = v.x * L.inv_scale;
        b = v.y * L.inv_scale;
    }
}
template <typename S>
__device__ __forceinline__ void st_pair(S* p, const Lat& L, typename St<S>::C a, typename St<S>::C b) {
    if constexpr (sizeof(S) == 8) {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
    } else if constexpr (sizeof(S) == 4) {
        *reinterpret_cast<float2*>(p) = make_float2(a, b);
    } else {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a * L.scale, b * L.scale);
    }
}

// Pre-collision populations of the node pair (x, x + 1) of row y, x even (Eq. 1, left
// side): one pair load per population, plus one scalar for the populations shifted in x
// (the value across the pair's edge), all issued before any is used.
template <typename S>
__device__ __forceinline__ void pull_pair(const S* __restrict__ src, const Lat& L, int x, int y,
                                          typename St<S>::C (&s0)[9], typename St<S>::C (&s1)[9]) {
    using C = typename St<S>::C;
    const int xm = x == 0 ? L.nx - 1 : x - 1, xp2 = x + 2 >= L.nx ? x + 2 - L.nx : x + 2;
    const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y + 1 == L.ny ? 0 : y + 1;
    const bool lo = L.walls && y == 0, hi = L.walls && y == L.ny - 1;
    C e[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const bool bounce = (ey(i) > 0 && lo) || (ey(i) < 0 && hi);
        const int sy = bounce ? y : (ey(i) > 0 ? ym : (ey(i) < 0 ? yp : y));
        const S* row = src + (long long)(bounce ? opp(i) : i) * L.plane + (long long)sy * L.pitch;
        ld_pair<S>(row + x, L, s0[i], s1[i]);
        e[i] = C(0);
        if (!bounce && ex(i) == 1) e[i] = St<S>::ldc(row + xm, L);
        if (!bounce && ex(i) == -1) e[i] = St<S>::ldc(row + xp2, L);
    }
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const bool bounce = (ey(i) > 0 && lo) || (ey(i) < 0 && hi);
        if (bounce) {
            const int j = opp(i);
            const C uw = ey(i) > 0 ? lat_c<C>(L.ub, L.ubf) : lat_c<C>(L.ut, L.utf);
            const C corr = C(6) * wgt<C>(j) * C(ex(j)) * uw;
            s0[i] -= corr;
            s1[i] -= corr;
        } else if (ex(i) == 1) {      // values at x - 1, x
            s1[i] = s0[i];
            s0[i] = e[i];
        } else if (ex(i) == -1) {     // values at x + 1, x + 2
            s0[i] = s1[i];
            s1[i] = e[i];
        }
    }
}

// Force-tile value at lattice node (x, y), or zero when the node is outside the tile.
// (x0w, y0w): tile origin wrapped into the lattice (y0w unwrapped between walls).
template <typename C>
__device__ __forceinline__ void tile_force(const Tile<C>& t, const Lat& L, int x0w, int y0w, int x, int y, C& fx,
                                           C& fy) {
    fx = C(0);
    fy = C(0);
    if (!t.use) return;
    int tx = x - x0w;
    if (tx < 0) tx += L.nx;
    int ty = y - y0w;
    if (!L.walls && ty < 0) ty += L.ny;
    if (tx < t.w && ty >= 0 && ty < t.h) {
        const int k = ty * t.w + tx;
        fx = t.fx[k];
        fy = t.fy[k];
    }
}

template <typename S>
__device__ void run_case(const BatchDev& d, int c, int nsteps, const CapSmem& sm, int tile_cells, int max_n) {
    using C = typename St<S>::C;
    BatchCase bc = d.cases[c];
    const Lat& L = bc.L;
    S* base = reinterpret_cast<S*>(d.pops) + bc.pops;
    const int n = bc.n, off = bc.off;
    const bool caps = n >= 3 && n <= max_n;
    const CapsuleParams P = d.nd.caps[c];   // membrane constants and the stress-free area
    // ring state in shared memory for the whole launch: X in sm.X, X^{n-1} in sm.ext,
    // the last interpolated velocity in sm.xd
    if (caps) {
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            sm.X[v] = d.nd.X[off + v];
            sm.ext[v] = d.nd.Xm1[off + v];
            sm.xd[v] = d.nd.uv[off + v];
        }
    }
    __syncthreads();
    int cur = bc.cur;
    int age = bc.age;
    bool ok = true, stable = true;
    const C gx = lat_c<C>(L.gx, L.gxf), gy = lat_c<C>(L.gy, L.gyf), om = lat_c<C>(L.omega, L.omegaf);
    for (int step = 0; step < nsteps; step++) {
        const S* src = base + (cur ? 9 * L.plane : 0);
        S* dst = base + (cur ? 0 : 9 * L.plane);
        Tile<C> t{};
        t.use = false;
        if (caps) {
            // i-iii: internal forces at X^n and their spread (c_v = 1) into the force tile
            t = make_tile<C>(sm, 0, n, 1, tile_cells, true, true);
            // a tile wider than the periodic lattice would alias lattice nodes
            if (t.use && (t.w > L.nx || (!L.walls && t.h > L.ny))) t.use = false;
            ok &= t.use;
            if (t.use) zero_forces<C>(t);
            // membrane terms (Eq. 11, 13, 14): in float for single-precision storage, as in
            // the single-case IB kernels (positions and the update stay double)
            constexpr bool F32 = sizeof(C) == 4;
            float fa = 0.0f;
            double A = 0.0;
            if constexpr (F32) {
                for (int v = threadIdx.x; v < n; v += blockDim.x)
                    vertex_terms_f(sm, P, d.nd, v == 0 ? n - 1 : v - 1, v, v + 1 == n ? 0 : v + 1, off + v);
                __syncthreads();
                float area2[1] = {0.0f};
                const double2 X0 = sm.X[0];
                for (int v = threadIdx.x; v < n; v += blockDim.x) {
                    const double2 Xv = sm.X[v];
                    const float2 e = ring_f(sm)[v].e;
                    area2[0] += (float)(Xv.x - X0.x) * e.y - (float)(Xv.y - X0.y) * e.x;
                }
                block_reduce<1, false>(area2, sm.red);
                // Eq. 14 factor k_a (1 - A/A0) p_ref / 2 from the difference A0 - A
                fa = (float)P.ka * (((float)P.A0 - 0.5f * area2[0]) / (6.0f * (float)P.A0));
            } else {
                double area2[1] = {0.0};
                for (int v = threadIdx.x; v < n; v += blockDim.x) area2[0] += ring_terms(sm, P, d.nd, v);
                block_reduce<1, false>(area2, sm.red);
                A = 0.5 * area2[0];
            }
            for (int v = threadIdx.x; v < n; v += blockDim.x) {
                double2 F;
                if constexpr (F32) {
                    const float2 Ff = internal_force_f(sm, v == 0 ? n - 1 : v - 1, v, v + 1 == n ? 0 : v + 1, fa);
                    F = make_double2(Ff.x, Ff.y);
                } else {
                    F = node_internal_force(sm, P, v, A);
                }
                if (t.use) {
                    const MlsW<C> m = mls_setup<C>(L, sm.X[v].x, sm.X[v].y);
                    ok &= m.ok && t.holds(m.cx, m.cy);
                    if (t.holds(m.cx, m.cy)) {
                        const C Fx = C(F.x), Fy = C(F.y);
#pragma unroll
                        for (int b = 0; b < 3; b++)
#pragma unroll
                            for (int a = 0; a < 3; a++) {
                                const C phi = m.phi(a, b);
                                const int k = t.index(m.cx + a - 1, m.cy + b - 1);
                                atomicAdd(t.fx + k, phi * Fx);
                                atomicAdd(t.fy + k, phi * Fy);
                            }
                    }
                }
                if (step == nsteps - 1) d.nd.Fint[off + v] = F;
            }
            __syncthreads();
        }
        // iv-vi: the lattice update of the whole case, with the membrane force inline. Each
        // thread walks nodes tid, tid + B, ... keeping (x, y) by carries instead of divisions.
        {
            const int x0w = t.use ? wrapi(t.x0, L.nx) : 0;
            const int y0w = t.use ? (L.walls ? t.y0 : wrapi(t.y0, L.ny)) : 0;
            if ((L.nx & 1) == 0) {
                // node pairs (x, x + 1), x even: walk pair tid, tid + B, ... by carries
                const int np = L.nx >> 1;
                const int dq = (int)blockDim.x / np, dr = (int)blockDim.x - dq * np;
                int y = (int)threadIdx.x / np, xp = (int)threadIdx.x - y * np;
                while (y < L.ny) {
                    const int x = 2 * xp;
                    C s0[9], s1[9];
                    pull_pair<S>(src, L, x, y, s0, s1);
                    C fx0, fy0, fx1, fy1;
                    tile_force<C>(t, L, x0w, y0w, x, y, fx0, fy0);
                    tile_force<C>(t, L, x0w, y0w, x + 1, y, fx1, fy1);
                    const C u0 = collide<C>(s0, gx + fx0, gy + fy0, om);
                    const C u1 = collide<C>(s1, gx + fx1, gy + fy1, om);
                    stable &= u0 < C(0.09) && u1 < C(0.09);
                    S* o = dst + (long long)y * L.pitch + x;
#pragma unroll
                    for (int i = 0; i < 9; i++) st_pair<S>(o + (long long)i * L.plane, L, s0[i], s1[i]);
                    xp += dr;
                    y += dq;
                    if (xp >= np) {
                        xp -= np;
                        y++;
                    }
                }
            } else {
            const int dq = (int)blockDim.x / L.nx, dr = (int)blockDim.x - dq * L.nx;
            int y = (int)threadIdx.x / L.nx, x = (int)threadIdx.x - y * L.nx;
            while (y < L.ny) {
                C s[9];
                pull_all<S, false>(src, L, x, y, s);   // plain loads: rewritten every step
                C fx, fy;
                tile_force<C>(t, L, x0w, y0w, x, y, fx, fy);
                const C usq = collide<C>(s, gx + fx, gy + fy, om);
                stable &= usq < C(0.09);
                S* o = dst + (long long)y * L.pitch + x;
#pragma unroll
                for (int i = 0; i < 9; i++) St<S>::st(o + (long long)i * L.plane, s[i], L);
                x += dr;
                y += dq;
                if (x >= L.nx) {
                    x -= L.nx;
                    y++;
                }
            }
            }
        }
        __syncthreads();  // the block's global stores are visible to the block after the barrier
        if (caps && t.use) {
            // vi-viii: moments of the new populations (with half the spread force) in the
            // tile, interpolation at X^n and the Eq. 25 advance
            const int cells = t.w * t.h;
            for (int k = threadIdx.x; k < cells; k += blockDim.x) {
                const int j = k / t.w, i = k - j * t.w;
                C q[9];
                pull_all<S, false>(dst, L, wrapi(t.x0 + i, L.nx), support_row(L, t.y0 + j), q);
                C drho, mx, my;
                moments<C>(q, drho, mx, my);
                const C inv = C(1) / (C(1) + drho);
                t.drho[k] = drho;
                t.ux[k] = (mx + C(0.5) * (gx + t.fx[k])) * inv;
                t.uy[k] = (my + C(0.5) * (gy + t.fy[k])) * inv;
            }
            __syncthreads();
            for (int v = threadIdx.x; v < n; v += blockDim.x) {
                const double2 Xv = sm.X[v];
                const MlsW<C> m = mls_setup<C>(L, Xv.x, Xv.y);
                InterpT<C> o;
                if (t.holds(m.cx, m.cy)) {
                    mls_apply<C, false>(m, [&](int a, int b) {
                        const int k = t.index(m.cx + a - 1, m.cy + b - 1);
                        Mom<C> r;
                        r.drho = t.drho[k];
                        r.ux = t.ux[k];
                        r.uy = t.uy[k];
                        return r;
                    }, o);
                } else {
                    ok = false;
                    o.ux = o.uy = C(0);
                }
                const double Ux = (double)o.ux, Uy = (double)o.uy;
                const double2 Xm = sm.ext[v];
                double2 Xn;
                if (age == 0) Xn = make_double2(Xv.x + Ux, Xv.y + Uy);
                else Xn = make_double2((2.0 / 3.0) * (2.0 * Xv.x - 0.5 * Xm.x + Ux),
                                       (2.0 / 3.0) * (2.0 * Xv.y - 0.5 * Xm.y + Uy));
                sm.ext[v] = Xv;
                sm.X[v] = Xn;
                sm.xd[v] = make_double2(Ux, Uy);
            }
            __syncthreads();
        }
        if (caps) age++;
        cur ^= 1;
    }
    if (caps) {
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            d.nd.X[off + v] = sm.X[v];
            d.nd.Xm1[off + v] = sm.ext[v];
            d.nd.uv[off + v] = sm.xd[v];
        }
    }
    if (threadIdx.x == 0) {
        d.cases[c].cur = cur;
        d.cases[c].age = age;
    }
    if (!ok) atomicOr(d.status, kStatSupport);
    if (__syncthreads_or(!stable)) {
        if (threadIdx.x == 0) atomicOr(d.status, kStatUnstable);
    }
}

template <typename S, int BS>
__global__ void __launch_bounds__(BS, 1024 / BS) k_batch(BatchDev d, int nsteps, int tile_cells, int max_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    const CapSmem sm = carve(smem, max_n);
    __shared__ int s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(d.queue, 1);
        __syncthreads();
        const int q = s_next;
        __syncthreads();
        if (q >= d.ncases) break;
        run_case<S>(d, d.order[q], nsteps, sm, tile_cells, max_n);
    }
}

template <typename C>
static size_t batch_smem(int max_n, int cells) {
    return ring_smem_bytes(max_n) + (size_t)cells * (3 * sizeof(C) + 2 * sizeof(C));
}

template <typename S>
static cudaError_t launch_batch(const BatchDev& d, int nsteps, int tile_cells, int max_n, int threads, int grid,
                                cudaStream_t s) {
    using C = typename St<S>::C;
    const size_t sh = batch_smem<C>(max_n, tile_cells);
    cudaError_t e = cudaSuccess;
#define LBMIB_BATCH(BS)                                                                             \
    e = cudaFuncSetAttribute(k_batch<S, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh); \
    if (e != cudaSuccess) return e;                                                                 \
    k_batch<S, BS><<<grid, BS, sh, s>>>(d, nsteps, tile_cells, max_n);
    if (threads == 256) {
        LBMIB_BATCH(256)
    } else if (threads == 512) {
        LBMIB_BATCH(512)
    } else {
        LBMIB_BATCH(1024)
    }
#undef LBMIB_BATCH
    return cudaGetLastError();
}

template <typename S>
static int batch_blocks_per_sm(int threads, int tile_cells, int max_n) {
    using C = typename St<S>::C;
    const size_t sh = batch_smem<C>(max_n, tile_cells);
    int nb = 0;
    if (threads == 256) {
        cudaFuncSetAttribute(k_batch<S, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<S, 256>, 256, sh);
    } else if (threads == 512) {
        cudaFuncSetAttribute(k_batch<S, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<S, 512>, 512, sh);
    } else {
        cudaFuncSetAttribute(k_batch<S, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<S, 1024>, 1024, sh);
    }
    return nb;
}

}  // namespace lbmib

using namespace lbmib;

namespace {

size_t sbytes(lbmib_storage s) { return s == LBMIB_FP64 ? 8 : (s == LBMIB_FP32 ? 4 : 2); }
size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct BatchLayout {
    std::vector<long long> pops;   // element offsets per case
    std::vector<int> pitch;
    size_t pops_bytes = 0;
    int nodes = 0, max_n = 0;
    long long max_N = 0;
    size_t off_cases, off_order, off_ctr, off_nodes[8], off_caps, off_obs, off_scratch, total;
};

bool case_ok(const lbmib_case& k) {
    return k.nx >= 3 && k.ny >= 3 && k.tau > 0.5 && (long long)k.nx * k.ny < (1LL << 31) &&
           (k.n == 0 || (k.xy && k.n >= 3 && k.n <= 1024 && k.node_mass > 0.0));
}

BatchLayout batch_layout(const lbmib_case* cases, int ncases, lbmib_storage st) {
    BatchLayout b;
    const size_t s = sbytes(st);
    long long elems = 0;
    for (int c = 0; c < ncases; c++) {
        const int pitch = (int)((cases[c].nx + 128 / s - 1) / (128 / s) * (128 / s));
        b.pitch.push_back(pitch);
        b.pops.push_back(elems);
        elems += 2LL * 9 * cases[c].ny * pitch;
        elems = (long long)(up256(elems * s) / s);
        b.nodes += cases[c].n;
        if (cases[c].n > b.max_n) b.max_n = cases[c].n;
        const long long N = (long long)cases[c].nx * cases[c].ny;
        if (N > b.max_N) b.max_N = N;
    }
    b.pops_bytes = up256(elems * s);
    size_t o = b.pops_bytes;
    auto take = [&](size_t bytes) { size_t r = o; o = up256(o + bytes); return r; };
    const size_t M = b.nodes > 0 ? b.nodes : 1;
    b.off_cases = take(sizeof(BatchCase) * ncases);
    b.off_order = take(sizeof(int) * ncases);
    b.off_ctr = take(sizeof(DevCounters));
    b.off_nodes[0] = take(M * sizeof(double2));  // X
    b.off_nodes[1] = take(M * sizeof(double2));  // Xm1
    b.off_nodes[2] = take(M * sizeof(double2));  // uv
    b.off_nodes[3] = take(M * sizeof(double2));  // Fint
    b.off_nodes[4] = take(M * sizeof(double));   // L0
    b.off_nodes[5] = take(M * sizeof(double));   // c0
    b.off_nodes[6] = take(M * sizeof(double));   // s0
    b.off_nodes[7] = take(M * sizeof(int));      // capid (for observables)
    b.off_caps = take(sizeof(CapsuleParams) * ncases);
    b.off_obs = take(8 * sizeof(double) * ncases);
    b.off_scratch = take(3 * sizeof(double) * (size_t)b.max_N);
    b.total = o;
    return b;
}

}  // namespace

struct lbmib_batch {
    lbmib_storage storage;
    int ncases = 0;
    cudaStream_t stream = nullptr;
    char* arena = nullptr;
    BatchLayout lay;
    BatchDev dev{};
    std::vector<BatchCase> host_cases;   // parameters (cur/age as last known)
    std::vector<CapsuleParams> caps;
    int tile_cells = 256;
    int threads = 512;
    int grid = 0;
    int sms = 0;
    long long launches = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = -1;
    std::string err;
};

namespace {

lbmib_status bfail(lbmib_batch* b, lbmib_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}
#define LBMIB_BCUDA(b, call)                                                                      \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return bfail((b), LBMIB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename F>
void by_st(lbmib_storage st, F&& f) {
    if (st == LBMIB_FP64) f(double{});
    else if (st == LBMIB_FP32) f(float{});
    else f(__half{});
}

lbmib_status batch_init_state(lbmib_batch* b, const lbmib_case* cases) {
    cudaStream_t s = b->stream;
    double* scratch = (double*)(b->arena + b->lay.off_scratch);
    for (int c = 0; c < b->ncases; c++) {
        const lbmib_case& k = cases[c];
        BatchCase& bc = b->host_cases[c];
        const size_t N = (size_t)k.nx * k.ny;
        const double* h[3] = {k.rho, k.ux, k.uy};
        for (int q = 0; q < 3; q++)
            if (h[q]) LBMIB_BCUDA(b, cudaMemcpyAsync(scratch + q * N, h[q], N * sizeof(double), cudaMemcpyHostToDevice, s));
        by_st(b->storage, [&](auto tag) {
            using S = decltype(tag);
            S* base = reinterpret_cast<S*>(b->arena) + bc.pops;
            launch_init<S>(base, bc.L, k.rho ? scratch : nullptr, k.ux ? scratch + N : nullptr,
                           k.uy ? scratch + 2 * N : nullptr, s);
        });
        b->launches++;
        LBMIB_BCUDA(b, cudaGetLastError());
        LBMIB_BCUDA(b, cudaStreamSynchronize(s));  // the scratch is reused by the next case
        bc.cur = 0;
        bc.age = 0;
        if (k.n > 0) {
            std::vector<double> xy(k.xy, k.xy + 2 * k.n);
            std::vector<double2> zero(k.n, make_double2(0.0, 0.0));
            const int off = bc.off;
            LBMIB_BCUDA(b, cudaMemcpyAsync(b->dev.nd.X + off, xy.data(), k.n * sizeof(double2), cudaMemcpyHostToDevice, s));
            LBMIB_BCUDA(b, cudaMemcpyAsync(b->dev.nd.Xm1 + off, xy.data(), k.n * sizeof(double2), cudaMemcpyHostToDevice, s));
            LBMIB_BCUDA(b, cudaMemcpyAsync(b->dev.nd.uv + off, zero.data(), k.n * sizeof(double2), cudaMemcpyHostToDevice, s));
            LBMIB_BCUDA(b, cudaStreamSynchronize(s));
        }
    }
    LBMIB_BCUDA(b, cudaMemcpyAsync(b->dev.cases, b->host_cases.data(), sizeof(BatchCase) * b->ncases,
                                   cudaMemcpyHostToDevice, s));
    LBMIB_BCUDA(b, cudaMemsetAsync(b->dev.status, 0, sizeof(unsigned), s));
    LBMIB_BCUDA(b, cudaStreamSynchronize(s));
    return LBMIB_OK;
}

lbmib_status batch_launch(lbmib_batch* b, int nsteps, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->dev.queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return bfail(b, LBMIB_ERR_CUDA, std::string("queue reset: ") + cudaGetErrorString(e));
    by_st(b->storage, [&](auto tag) {
        using S = decltype(tag);
        e = launch_batch<S>(b->dev, nsteps, b->tile_cells, b->lay.max_n > 0 ? b->lay.max_n : 1, b->threads, b->grid, s);
    });
    if (e != cudaSuccess) return bfail(b, LBMIB_ERR_CUDA, std::string("batched launch: ") + cudaGetErrorString(e));
    b->launches++;
    return LBMIB_OK;
}

// Resident CTAs per SM for the current CTA size (registers and shared memory).
int max_blocks_per_sm(lbmib_batch* b) {
    int per_sm = 1;
    by_st(b->storage, [&](auto tag) {
        using S = decltype(tag);
        per_sm = batch_blocks_per_sm<S>(b->threads, b->tile_cells, b->lay.max_n > 0 ? b->lay.max_n : 1);
    });
    return per_sm < 1 ? 1 : per_sm;
}

// Persistent grid: blocks_per_sm CTAs on every SM (0: as many as fit), at most one per case.
void set_grid(lbmib_batch* b, int blocks_per_sm = 0) {
    const int most = max_blocks_per_sm(b);
    const int per_sm = blocks_per_sm > 0 && blocks_per_sm < most ? blocks_per_sm : most;
    b->grid = per_sm * b->sms;
    if (b->grid > b->ncases) b->grid = b->ncases;
}

}  // namespace

extern "C" {

size_t lbmib_batch_arena_bytes(const lbmib_case* cases, int ncases, lbmib_storage storage) {
    if (!cases || ncases <= 0 || (storage != LBMIB_FP64 && storage != LBMIB_FP32 && storage != LBMIB_FP16)) return 0;
    for (int c = 0; c < ncases; c++)
        if (!case_ok(cases[c])) return 0;
    return batch_layout(cases, ncases, storage).total;
}

lbmib_status lbmib_batch_create(const lbmib_case* cases, int ncases, lbmib_storage storage, void* d_arena,
                                size_t arena_bytes, void* cuda_stream, int autotune_steps, lbmib_batch** out) {
    if (!out) return LBMIB_ERR_ARG;
    *out = nullptr;
    const size_t need = lbmib_batch_arena_bytes(cases, ncases, storage);
    if (need == 0 || !d_arena || ((uintptr_t)d_arena % 256) != 0) return LBMIB_ERR_ARG;
    if (arena_bytes < need) return LBMIB_ERR_OOM;
    lbmib_batch* b = new lbmib_batch();
    b->storage = storage;
    b->ncases = ncases;
    b->stream = (cudaStream_t)cuda_stream;
    b->arena = (char*)d_arena;
    b->lay = batch_layout(cases, ncases, storage);
    const BatchLayout& lay = b->lay;
    char* a = b->arena;
    b->dev.pops = a;
    b->dev.cases = (BatchCase*)(a + lay.off_cases);
    b->dev.order = (const int*)(a + lay.off_order);
    DevCounters* ctr = (DevCounters*)(a + lay.off_ctr);
    b->dev.queue = &ctr->count[0];
    b->dev.status = &ctr->status;
    b->dev.nd.X = (double2*)(a + lay.off_nodes[0]);
    b->dev.nd.Xm1 = (double2*)(a + lay.off_nodes[1]);
    b->dev.nd.uv = (double2*)(a + lay.off_nodes[2]);
    b->dev.nd.Fint = (double2*)(a + lay.off_nodes[3]);
    b->dev.nd.Fext = nullptr;
    b->dev.nd.L0 = (double*)(a + lay.off_nodes[4]);
    b->dev.nd.c0 = (double*)(a + lay.off_nodes[5]);
    b->dev.nd.s0 = (double*)(a + lay.off_nodes[6]);
    b->dev.nd.capid = (int*)(a + lay.off_nodes[7]);
    b->dev.nd.age = nullptr;
    b->dev.nd.caps = (const CapsuleParams*)(a + lay.off_caps);
    b->dev.nd.count = lay.nodes;
    b->dev.ncases = ncases;
    cudaDeviceProp prop{};
    int devid = 0;
    cudaGetDevice(&devid);
    cudaGetDeviceProperties(&prop, devid);
    b->sms = prop.multiProcessorCount;

    // per-case lattice descriptions, vertex ranges and membrane references
    std::vector<double> L0s, c0s, s0s;
    std::vector<int> capid;
    double max_extent = 0.0;
    int off = 0;
    for (int c = 0; c < ncases; c++) {
        const lbmib_case& k = cases[c];
        BatchCase bc{};
        Lat& L = bc.L;
        L.nx = k.nx;
        L.ny = k.ny;
        L.pitch = lay.pitch[c];
        L.plane = (long long)k.ny * L.pitch;
        L.walls = k.walls ? 1 : 0;
        L.tau = k.tau;
        L.omega = 1.0 / k.tau;
        L.ub = k.walls ? k.u_bottom : 0.0;
        L.ut = k.walls ? k.u_top : 0.0;
        L.gx = k.gx;
        L.gy = k.gy;
        L.scale = storage == LBMIB_FP16 ? 1024.0f : 1.0f;
        L.inv_scale = 1.0f / L.scale;
        L.nu = (k.tau - 0.5) / 3.0;
        L.gxf = (float)L.gx;
        L.gyf = (float)L.gy;
        L.omegaf = (float)L.omega;
        L.ubf = (float)L.ub;
        L.utf = (float)L.ut;
        bc.pops = lay.pops[c];
        bc.off = off;
        bc.n = k.n;
        CapsuleParams P{off, k.n, k.k_s, k.k_b, k.k_a, k.node_mass, 0.0, 0.0};
        if (k.n > 0) {
            double a2 = 0.0, per = 0.0, x0 = k.xy[0], x1 = k.xy[0], y0 = k.xy[1], y1 = k.xy[1];
            for (int v = 0; v < k.n; v++) {
                const int r = (v + 1) % k.n, l = (v + k.n - 1) % k.n;
                const double dx = k.xy[2 * r] - k.xy[2 * v], dy = k.xy[2 * r + 1] - k.xy[2 * v + 1];
                const double len = std::sqrt(dx * dx + dy * dy);
                L0s.push_back(len);
                per += len;
                const double ax = k.xy[2 * v] - k.xy[2 * l], ay = k.xy[2 * v + 1] - k.xy[2 * l + 1];
                const double nrm = std::sqrt((ax * ax + ay * ay) * (dx * dx + dy * dy));
                c0s.push_back((ax * dx + ay * dy) / nrm);
                s0s.push_back((ax * dy - ay * dx) / nrm);
                a2 += (k.xy[2 * v] - k.xy[0]) * (k.xy[2 * r + 1] - k.xy[1]) -
                      (k.xy[2 * r] - k.xy[0]) * (k.xy[2 * v + 1] - k.xy[1]);
                capid.push_back(c);
                x0 = std::fmin(x0, k.xy[2 * v]); x1 = std::fmax(x1, k.xy[2 * v]);
                y0 = std::fmin(y0, k.xy[2 * v + 1]); y1 = std::fmax(y1, k.xy[2 * v + 1]);
            }
            P.A0 = 0.5 * a2;
            P.P0 = per;
            if (!(P.A0 > 0.0)) {
                delete b;
                return LBMIB_ERR_ARG;  // rings must be counter-clockwise
            }
            // the ring's bounding-box side: a tile of 1.5 (side + 8)^2 cells leaves room for
            // the deformation and rotation of a capsule in shear
            max_extent = std::fmax(max_extent, std::fmax(x1 - x0, y1 - y0));
        }
        off += k.n;
        b->host_cases.push_back(bc);
        b->caps.push_back(P);
    }
    b->tile_cells = tile_budget(lay.max_n > 0 ? lay.max_n : 1, max_extent);
    // processing order: largest lattice first (longest-processing-time scheduling)
    std::vector<int> order(ncases);
    for (int c = 0; c < ncases; c++) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (long long)cases[x].nx * cases[x].ny > (long long)cases[y].nx * cases[y].ny;
    });
    cudaStream_t s = b->stream;
    cudaError_t e = cudaMemcpyAsync((void*)b->dev.order, order.data(), sizeof(int) * ncases, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && lay.nodes > 0) {
        e = cudaMemcpyAsync(b->dev.nd.L0, L0s.data(), lay.nodes * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->dev.nd.c0, c0s.data(), lay.nodes * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->dev.nd.s0, s0s.data(), lay.nodes * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->dev.nd.capid, capid.data(), lay.nodes * sizeof(int), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void*)b->dev.nd.caps, b->caps.data(), sizeof(CapsuleParams) * ncases, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, sizeof(DevCounters), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete b;
        return LBMIB_ERR_CUDA;
    }
    lbmib_status st = batch_init_state(b, cases);
    if (st != LBMIB_OK) {
        delete b;
        return st;
    }
    // autotuner: time every launch shape (threads per CTA x resident CTAs per SM) for a
    // few steps, keep the fastest, then restart every case from its initial state
    b->threads = 512;
    set_grid(b);
    if (autotune_steps > 0) {
        const int cand[3] = {256, 512, 1024};
        float best = 1e30f;
        int best_t = 512, best_g = b->grid;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int t : cand) {
            b->threads = t;
            const int most = max_blocks_per_sm(b);
            int prev = -1;
            for (int per_sm = 1; per_sm <= most; per_sm++) {
                set_grid(b, per_sm);
                if (b->grid == prev) break;   // capped at one CTA per case
                prev = b->grid;
                cudaEventRecord(e0, s);
                st = batch_launch(b, autotune_steps, s);
                cudaEventRecord(e1, s);
                if (st != LBMIB_OK || cudaStreamSynchronize(s) != cudaSuccess) continue;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_t = t;
                    best_g = b->grid;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->threads = best_t;
        b->grid = best_g;
        st = batch_init_state(b, cases);
        if (st != LBMIB_OK) {
            delete b;
            return st;
        }
    }
    *out = b;
    return LBMIB_OK;
}

void lbmib_batch_destroy(lbmib_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    delete b;
}

const char* lbmib_batch_last_error(const lbmib_batch* b) { return b ? b->err.c_str() : "null batch"; }

lbmib_status lbmib_batch_step(lbmib_batch* b, long long nsteps) {
    if (!b || nsteps < 0 || nsteps > (1LL << 30)) return LBMIB_ERR_ARG;
    if (nsteps == 0) return LBMIB_OK;
    if (!b->graph || b->graph_steps != (int)nsteps) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaStream_t cs;
        LBMIB_BCUDA(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        lbmib_status st = LBMIB_OK;
        if (e == cudaSuccess) {
            st = batch_launch(b, (int)nsteps, cs);
            b->launches--;  // captured, not launched
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cs, &g);
            if (e == cudaSuccess && st == LBMIB_OK) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
        }
        cudaStreamDestroy(cs);
        if (st != LBMIB_OK) return st;
        if (e != cudaSuccess) return bfail(b, LBMIB_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        b->graph_steps = (int)nsteps;
    }
    LBMIB_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    b->launches++;
    for (auto& c : b->host_cases) {
        if ((nsteps & 1) != 0) c.cur ^= 1;
        if (c.n > 0) c.age += (int)nsteps;
    }
    return LBMIB_OK;
}

lbmib_status lbmib_batch_sync(lbmib_batch* b) {
    if (!b) return LBMIB_ERR_ARG;
    LBMIB_BCUDA(b, cudaStreamSynchronize(b->stream));
    unsigned st = 0;
    LBMIB_BCUDA(b, cudaMemcpy(&st, b->dev.status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st & kStatUnstable) return bfail(b, LBMIB_ERR_UNSTABLE, "unstable lattice in a batched case");
    if (st & kStatSupport) return bfail(b, LBMIB_ERR_SUPPORT, "a batched capsule left its channel or its tile");
    return LBMIB_OK;
}

lbmib_status lbmib_batch_read_populations(lbmib_batch* b, int c, double* f) {
    if (!b || c < 0 || c >= b->ncases || !f) return LBMIB_ERR_ARG;
    LBMIB_BCUDA(b, cudaStreamSynchronize(b->stream));
    const BatchCase& bc = b->host_cases[c];
    const size_t N = (size_t)bc.L.nx * bc.L.ny;
    double* scratch = (double*)(b->arena + b->lay.off_scratch);
    for (int i0 = 0; i0 < 9; i0 += 3) {
        by_st(b->storage, [&](auto tag) {
            using S = decltype(tag);
            const S* base = reinterpret_cast<const S*>(b->arena) + bc.pops + (bc.cur ? 9 * bc.L.plane : 0);
            launch_populations<S>(base, bc.L, OpenBC{}, i0, scratch, b->stream);
        });
        LBMIB_BCUDA(b, cudaGetLastError());
        LBMIB_BCUDA(b, cudaMemcpyAsync(f + i0 * N, scratch, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        LBMIB_BCUDA(b, cudaStreamSynchronize(b->stream));
    }
    return lbmib_batch_sync(b);
}

lbmib_status lbmib_batch_read_capsule(lbmib_batch* b, int c, double* xy, double* vel) {
    if (!b || c < 0 || c >= b->ncases) return LBMIB_ERR_ARG;
    const BatchCase& bc = b->host_cases[c];
    if (bc.n == 0) return LBMIB_OK;
    if (xy) LBMIB_BCUDA(b, cudaMemcpyAsync(xy, b->dev.nd.X + bc.off, bc.n * sizeof(double2), cudaMemcpyDeviceToHost, b->stream));
    if (vel) LBMIB_BCUDA(b, cudaMemcpyAsync(vel, b->dev.nd.uv + bc.off, bc.n * sizeof(double2), cudaMemcpyDeviceToHost, b->stream));
    return lbmib_batch_sync(b);
}

lbmib_status lbmib_batch_observables(lbmib_batch* b, double* out) {
    if (!b || !out) return LBMIB_ERR_ARG;
    double* obs = (double*)(b->arena + b->lay.off_obs);
    LBMIB_BCUDA(b, cudaMemsetAsync(obs, 0, 8 * sizeof(double) * b->ncases, b->stream));
    launch_observables(b->dev.nd, b->ncases, b->lay.max_n > 0 ? b->lay.max_n : 1, obs, b->stream);
    LBMIB_BCUDA(b, cudaGetLastError());
    LBMIB_BCUDA(b, cudaMemcpyAsync(out, obs, 8 * sizeof(double) * b->ncases, cudaMemcpyDeviceToHost, b->stream));
    return lbmib_batch_sync(b);
}

lbmib_status lbmib_batch_config(const lbmib_batch* b, int* threads, int* grid, int* tile_cells) {
    if (!b) return LBMIB_ERR_ARG;
    if (threads) *threads = b->threads;
    if (grid) *grid = b->grid;
    if (tile_cells) *tile_cells = b->tile_cells;
    return LBMIB_OK;
}

}  // extern "C"
