// Host-side declarations of the kernel launchers (internal to the library).
#pragma once

#include "lbmib_internal.cuh"

namespace lbmib {

// State of a rigid particle (Section 2.3.1, Eq. 17-20): {c_x, c_y, theta, u_x, u_y,
// omega} at step n and at n - 1 (c the area centroid), mass, moment of inertia about c,
// and the last fluid load {F_x, F_y, M}.
struct RigidBody {
    double body[6], prev[6];
    double mass, inertia;
    double load[3];
};

// Membrane vertex state, structure of arrays over all vertices of all capsules.
struct Nodes {
    double2* X;      // X^n
    double2* Xm1;    // X^{n-1}
    double2* uv;     // node velocity (Dynamic: Eq. 24; Kinematic: interpolated)
    double2* Fint;   // last internal force (Eq. 22)
    double2* Fext;   // last external force (Eq. 15-16)
    double2* U;      // Dynamic: fluid velocity at X^n interpolated by the step's forcing
                     // (step 1), the tentative velocity of the step's Eq. 23
    double* L0;      // stress-free length of element v (v -> v+1)
    double* c0;      // cos(theta_0) at vertex v
    double* s0;      // sin(theta_0) at vertex v
    int* age;        // steps taken since the vertex's history started
    int* capid;      // capsule of the vertex
    const CapsuleParams* caps;
    int count;       // vertices in use
    double2* Flc;    // optional (null): c_l F_l of the last Dynamic spread, per vertex
    void* mls;       // MLS shape functions of each vertex at X^n (MlsW of the compute type),
                     // written by the spread kernels, read by the node update of the step
    double2* Fpp;    // optional (null): capsule-capsule repulsion at X^n (Eq. 27)
    RigidBody* rb;   // per capsule; read for capsules with CapsuleParams::rigid
    double2* R0;     // per vertex of a rigid particle: offset from c in the body frame
};

// Neighbour grid of the capsule-capsule repulsion: capsules hashed by the coarse cell of
// their bounding-box centre into fixed-capacity buckets.
struct RepGrid {
    double cellx, celly;   // coarse cell sides (>= largest capsule extent + cut-off)
    int ncx, ncy;      // coarse cells along x and y
    int nbuckets;      // power of two
    int* count;        // per bucket (cleared every step)
    int* slot;         // nbuckets x kRepSlots capsule ids
    int* cellof;       // per capsule: its coarse cell (iy * ncx + ix)
    double* box;       // per capsule: min x, min y, max x, max y
    double rc, coeff;  // cut-off and coefficient of Eq. 27
};
constexpr int kRepSlots = 16;

// Touched-cell bookkeeping for the spread of one step.
struct Spread {
    double* fib;     // force buffer written this step (fx[N] then fy[N])
    int* list;       // unique touched cells of this step
    int* count;      // length of list
    int capacity;    // entries the list can hold
    unsigned* status;
};

// lattice.cu
template <typename S>
void launch_collide_stream(const void* src, void* dst, const Lat& L, unsigned* status, int variant,
                           cudaStream_t s);
// force the listed nodes in place (their unforced post-collision populations in dst)
template <typename S>
void launch_patch(void* dst, const Lat& L, const double* fib_c, const int* list_c, double* fib_p,
                  const int* list_p, int* mark, DevCounters* ctr, int c, int capacity, long long vertices,
                  cudaStream_t s);
// open channel: Zou-He inlet and outlet columns, after launch_collide_stream on its output
template <typename S>
void launch_open_columns(const void* src, void* dst, const Lat& L, const OpenBC& ob, unsigned* status,
                         cudaStream_t s);
template <typename S>
void launch_init(void* dst, const Lat& L, const double* rho, const double* ux, const double* uy, cudaStream_t s);
template <typename S>
void launch_macros(const void* src, const Lat& L, const OpenBC& ob, const double* fib, double* rho, double* ux, double* uy,
                   cudaStream_t s);
template <typename S>
void launch_populations(const void* src, const Lat& L, const OpenBC& ob, int i0, double* out, cudaStream_t s);

// ib.cu. The capsule kernels run `arcs` CTAs per capsule (1..kMaxArcs), each on an even
// share of the ring.
constexpr int kHalo = 2;       // neighbour slots staged on each side of an arc
constexpr int kMaxArcs = 8;    // portable thread-block cluster size
// staged vertex slots per CTA for rings of at most max_n vertices in `arcs` arcs
__host__ __device__ inline int arc_slots(int max_n, int arcs) { return (max_n + arcs - 1) / arcs + 2 * kHalo; }
template <typename S>
void launch_dyn_force_spread(const void* src, const Lat& L, Nodes nd, int ncaps, int max_n,
                             int arcs, int cells, bool rigid, Spread sp, unsigned* status, cudaStream_t s);
// the node update of the capsules, then (rigid: the context holds rigid particles) that
// of the rigid particles
template <typename S>
void launch_dyn_update(const void* dst, const Lat& L, Nodes nd, int ncaps, int max_n,
                       int arcs, int cells, bool rigid, int* reset_count, unsigned* status, cudaStream_t s);
// the node update of step n and the force and spread of step n+1 in one kernel (one CTA
// per capsule, no rigid particles), spreading through sp_next
template <typename S>
void launch_dyn_update_spread(const void* dst, const Lat& L, Nodes nd, int ncaps, int max_n,
                              int cells, Spread sp_next, unsigned* status, cudaStream_t s);
void launch_kin_force_spread(const Lat& L, Nodes nd, int ncaps, int max_n, int arcs, int cells, Spread sp,
                             unsigned* status, bool fp64_weights, cudaStream_t s);
template <typename S>
void launch_kin_advance(const void* dst, const Lat& L, const double* fib_cur, Nodes nd, int ncaps, int max_n,
                        int arcs, int cells, int* reset_count, unsigned* status, cudaStream_t s);
// the Kinematic node advance of step n and the force and spread of step n+1 in one kernel
// (one CTA per capsule, no rigid particles, no repulsion), spreading through sp_next
template <typename S>
void launch_kin_advance_spread(const void* dst, const Lat& L, const double* fib_cur, Nodes nd, int ncaps, int max_n,
                               int cells, Spread sp_next, unsigned* status, cudaStream_t s);
void launch_observables(Nodes nd, int ncaps, int max_n, double* out, cudaStream_t s);
template <typename S>
void launch_interp_points(const void* src, const Lat& L, const double* fib, const double2* pts, int n,
                          double* out, unsigned* status, cudaStream_t s);
// repulsion.cu
void launch_repulsion(const Lat& L, Nodes nd, int ncaps, int max_n, int arcs, RepGrid g, unsigned* status,
                      cudaStream_t s);
size_t capsule_smem_bytes(int max_n);
// tile cells per CTA for `slots` staged vertices and boxes of about `extent` across
// (`tight`: no allowance for rotation and deformation)
int tile_budget(int slots, double extent, bool tight = false);
void set_capsule_smem_limits(int slots, int tile_cells);

}  // namespace lbmib
