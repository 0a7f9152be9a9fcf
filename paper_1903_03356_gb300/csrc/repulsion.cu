// Capsule-capsule repulsion (Section 3.4, Eq. 27): on vertex 1 of a capsule, from every
// vertex 2 of another capsule closer than the cut-off r_c,
//   F_1 += 1e-4 / (8 sqrt 2) sqrt(dx / d_12^5) n_1^-   (dx = 1),
// with n_1^- the inward normal at vertex 1: the negated, normalised sum of the outward
// normals (dy, -dx)/l of the two elements that meet there. Distances along periodic
// axes are minimum images (x is not periodic in an open channel).
//
// Broad phase: each capsule's bounding box, and its coarse cell (side >= largest capsule
// extent + r_c, so interacting capsules sit in neighbouring cells), hashed into
// fixed-capacity buckets. Narrow phase: one CTA per arc of a ring stages the arc and,
// for each capsule of the 3 x 3 neighbouring cells whose box comes within r_c of the
// arc's box, stages that ring with the boxes of its 32-vertex chunks and sums the pair
// forces over the chunks within r_c of each vertex. A capsule is accepted only from its
// own cell, so hash collisions cannot count it twice.
#include "ring.cuh"

namespace lbmib {
namespace {

__device__ __forceinline__ double min_image(double d, double P) {
    return P > 0.0 ? d - P * floor(d / P + 0.5) : d;
}

__device__ __forceinline__ int bucket_of(int ix, int iy, int nb) {
    unsigned h = (unsigned)ix * 73856093u ^ (unsigned)iy * 19349663u;
    return (int)(h & (unsigned)(nb - 1));
}

// Bounding box, coarse cell and bucket entry of every capsule (one CTA per capsule).
__global__ void __launch_bounds__(128) k_rep_bin(Lat L, Nodes nd, int max_n, RepGrid g, unsigned* status) {
    __shared__ double red[32 * 8];
    const int c = blockIdx.x;
    const CapsuleParams P = nd.caps[c];
    if (P.n < 3 || P.n > max_n) return;
    double r[4] = {1e300, 1e300, 1e300, 1e300};   // min x, min y, -max x, -max y
    for (int v = threadIdx.x; v < P.n; v += blockDim.x) {
        const double2 X = nd.X[P.off + v];
        r[0] = fmin(r[0], X.x);
        r[1] = fmin(r[1], X.y);
        r[2] = fmin(r[2], -X.x);
        r[3] = fmin(r[3], -X.y);
    }
    block_reduce<4, true>(r, red);
    if (threadIdx.x != 0) return;
    const double b[4] = {r[0], r[1], -r[2], -r[3]};
    for (int k = 0; k < 4; k++) g.box[4 * c + k] = b[k];
    const bool sane = fabs(b[0]) < 1e9 && fabs(b[1]) < 1e9 && fabs(b[2]) < 1e9 && fabs(b[3]) < 1e9;
    const double cx = sane ? 0.5 * (b[0] + b[2]) : 0.0, cy = sane ? 0.5 * (b[1] + b[3]) : 0.0;
    if (!sane || b[2] - b[0] > g.cellx - g.rc || b[3] - b[1] > g.celly - g.rc) atomicOr(status, kStatGrid);
    int ix = (int)floor(cx / g.cellx) % g.ncx;
    if (ix < 0) ix += g.ncx;
    int iy = (int)floor(cy / g.celly);
    if (L.walls) iy = iy < 0 ? 0 : (iy >= g.ncy ? g.ncy - 1 : iy);
    else {
        iy %= g.ncy;
        if (iy < 0) iy += g.ncy;
    }
    g.cellof[c] = iy * g.ncx + ix;
    const int h = bucket_of(ix, iy, g.nbuckets);
    const int k = atomicAdd(&g.count[h], 1);
    if (k < kRepSlots) g.slot[(size_t)h * kRepSlots + k] = c;
    else atomicOr(status, kStatGrid);
}

constexpr int kRepChunk = 32;        // vertices per chunk box of a neighbour's ring
// Slack of the box tests: a box test may keep a pair that the exact test then drops,
// never the reverse, whatever the rounding of the box arithmetic.
constexpr double kRepSlack = 1e-9;

// Distance along one axis from coordinate x to the box [lo, hi] (0 inside), through the
// periodic images when P > 0.
__device__ __forceinline__ double axis_gap(double x, double lo, double hi, double P) {
    return fabs(min_image(x - 0.5 * (lo + hi), P)) - 0.5 * (hi - lo);
}

// Eq. 27 forces on the vertices of one arc of a ring: CTA blockIdx.x = c * arcs + rank
// owns the same share of capsule c's ring as in the immersed-boundary kernels. Each
// neighbour capsule whose box comes within r_c of the arc's box is staged with boxes of
// its 32-vertex chunks; a vertex then scans only the chunks within r_c of it.
__global__ void __launch_bounds__(128) k_repulsion(Lat L, Nodes nd, int max_n, int arcs, RepGrid g) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int slots = (max_n + arcs - 1) / arcs;
    double2* own = reinterpret_cast<double2*>(smem);   // own arc: vertex v0 - 1 + li in slot li
    double2* nrm = own + slots + 2;                    // inward normal of own vertex k
    double2* oth = nrm + slots;                        // a neighbour's ring
    double* cbox = reinterpret_cast<double*>(oth + max_n);   // its chunk boxes (min x, min y, max x, max y)
    __shared__ double red[32 * 8];
    const int c = blockIdx.x / arcs, rank = blockIdx.x - c * arcs;
    const CapsuleParams P = nd.caps[c];
    if (P.n < 3 || P.n > max_n) return;
    const int n = P.n, chunk = (n + arcs - 1) / arcs, v0 = rank * chunk, m = min(n - v0, chunk);
    if (m <= 0) return;
    const double px = L.inflow ? 0.0 : (double)L.nx, py = L.walls ? 0.0 : (double)L.ny;
    for (int li = threadIdx.x; li < m + 2; li += blockDim.x) own[li] = nd.X[P.off + (v0 - 1 + li + n) % n];
    __syncthreads();
    double r[4] = {1e300, 1e300, 1e300, 1e300};   // the arc's box: min x, min y, -max x, -max y
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const double2 Xl = own[k], Xv = own[k + 1], Xr = own[k + 2];
        const double ax = Xv.x - Xl.x, ay = Xv.y - Xl.y, bx = Xr.x - Xv.x, by = Xr.y - Xv.y;
        const double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
        const double nx = ay / la + by / lb, ny = -ax / la - bx / lb;
        const double ln = sqrt(nx * nx + ny * ny);
        nrm[k] = make_double2(-nx / ln, -ny / ln);
        r[0] = fmin(r[0], Xv.x);
        r[1] = fmin(r[1], Xv.y);
        r[2] = fmin(r[2], -Xv.x);
        r[3] = fmin(r[3], -Xv.y);
    }
    block_reduce<4, true>(r, red);
    const double mb[4] = {r[0], r[1], -r[2], -r[3]};
    const double reach = g.rc + kRepSlack;
    const int cell = g.cellof[c], ix = cell % g.ncx, iy = cell / g.ncx;
    double facc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // own vertices threadIdx.x + 128 k, k < 8
    const int nxs = g.ncx < 3 ? g.ncx : 3, nys = (!L.walls && g.ncy < 3) ? g.ncy : 3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int sy = 0; sy < nys; sy++) {
        int jy = iy + sy - (nys == 3 ? 1 : 0);
        if (L.walls && (jy < 0 || jy >= g.ncy)) continue;
        if (!L.walls) jy = ((jy % g.ncy) + g.ncy) % g.ncy;
        for (int sx = 0; sx < nxs; sx++) {
            const int jx = ((ix + sx - (nxs == 3 ? 1 : 0)) % g.ncx + g.ncx) % g.ncx;
            const int h = bucket_of(jx, jy, g.nbuckets);
            const int cnt = min(g.count[h], kRepSlots);
            for (int e = 0; e < cnt; e++) {
                const int o = g.slot[(size_t)h * kRepSlots + e];
                if (o == c || g.cellof[o] != jy * g.ncx + jx) continue;   // self, or another cell's entry
                const double* ob = g.box + 4 * o;
                // boxes closer than r_c (minimum image between their centres)
                const double gx = fabs(min_image(0.5 * (ob[0] + ob[2]) - 0.5 * (mb[0] + mb[2]), px)) -
                                  0.5 * ((ob[2] - ob[0]) + (mb[2] - mb[0]));
                const double gy = fabs(min_image(0.5 * (ob[1] + ob[3]) - 0.5 * (mb[1] + mb[3]), py)) -
                                  0.5 * ((ob[3] - ob[1]) + (mb[3] - mb[1]));
                if (gx >= reach || gy >= reach) continue;
                const CapsuleParams Q = nd.caps[o];
                if (Q.n < 3 || Q.n > max_n) continue;
                const int nch = (Q.n + kRepChunk - 1) / kRepChunk;
                __syncthreads();
                for (int w = threadIdx.x; w < Q.n; w += blockDim.x) oth[w] = nd.X[Q.off + w];
                __syncthreads();
                for (int ch = warp; ch < nch; ch += nwarps) {
                    const int w = ch * kRepChunk + lane;
                    const double2 X = oth[w < Q.n ? w : ch * kRepChunk];
                    double b0 = X.x, b1 = X.y, b2 = X.x, b3 = X.y;
                    for (int sh = 16; sh > 0; sh >>= 1) {
                        b0 = fmin(b0, __shfl_xor_sync(0xffffffffu, b0, sh));
                        b1 = fmin(b1, __shfl_xor_sync(0xffffffffu, b1, sh));
                        b2 = fmax(b2, __shfl_xor_sync(0xffffffffu, b2, sh));
                        b3 = fmax(b3, __shfl_xor_sync(0xffffffffu, b3, sh));
                    }
                    if (lane == 0) {
                        cbox[4 * ch] = b0;
                        cbox[4 * ch + 1] = b1;
                        cbox[4 * ch + 2] = b2;
                        cbox[4 * ch + 3] = b3;
                    }
                }
                __syncthreads();
                for (int k = 0, v = threadIdx.x; v < m && k < 8; k++, v += blockDim.x) {
                    const double2 Xv = own[v + 1];
                    if (axis_gap(Xv.x, ob[0], ob[2], px) >= reach || axis_gap(Xv.y, ob[1], ob[3], py) >= reach)
                        continue;
                    double f = 0.0;
                    for (int ch = 0; ch < nch; ch++) {
                        const double* cb = cbox + 4 * ch;
                        if (axis_gap(Xv.x, cb[0], cb[2], px) >= reach || axis_gap(Xv.y, cb[1], cb[3], py) >= reach)
                            continue;
                        const int w1 = min(Q.n, (ch + 1) * kRepChunk);
                        for (int w = ch * kRepChunk; w < w1; w++) {
                            const double dx = min_image(Xv.x - oth[w].x, px), dy = min_image(Xv.y - oth[w].y, py);
                            const double d2 = dx * dx + dy * dy;
                            if (d2 < g.rc * g.rc) f += g.coeff * rsqrt(d2 * d2 * sqrt(d2));   // coeff d^{-5/2}
                        }
                    }
                    facc[k] += f;
                }
            }
        }
    }
    for (int k = 0, v = threadIdx.x; v < m && k < 8; k++, v += blockDim.x)
        nd.Fpp[P.off + v0 + v] = make_double2(facc[k] * nrm[v].x, facc[k] * nrm[v].y);
}

}  // namespace

void launch_repulsion(const Lat& L, Nodes nd, int ncaps, int max_n, int arcs, RepGrid g, unsigned* status,
                      cudaStream_t s) {
    cudaMemsetAsync(g.count, 0, sizeof(int) * (size_t)g.nbuckets, s);
    k_rep_bin<<<ncaps, 128, 0, s>>>(L, nd, max_n, g, status);
    const size_t slots = (size_t)((max_n + arcs - 1) / arcs);
    const size_t sh = (2 * slots + 2 + (size_t)max_n) * sizeof(double2) +
                      4 * sizeof(double) * (size_t)((max_n + kRepChunk - 1) / kRepChunk);
    cudaFuncSetAttribute(k_repulsion, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    k_repulsion<<<ncaps * arcs, 128, sh, s>>>(L, nd, max_n, arcs, g);
}

}  // namespace lbmib
