// Internal declarations of the GB300 PIC library: host mesh, device record layouts,
// precision policies and kernel launchers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pic.h"

namespace pic {

// ---------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------
void set_error(const char *fmt, ...);

// Handlers closing the function-try-block of every status-returning entry point, so that
// no C++ exception (a failed host allocation, a thread that cannot start) crosses the C
// ABI: the call returns a status and leaves its message instead.
#define PIC_CATCH(name)                                                    \
    catch (const std::bad_alloc &) {                                       \
        ::pic::set_error("%s: out of host memory", name);                  \
        return PIC_ERR_OOM;                                                \
    }                                                                      \
    catch (const std::exception &ex__) {                                   \
        ::pic::set_error("%s: %s", name, ex__.what());                     \
        return PIC_ERR_ARG;                                                \
    }                                                                      \
    catch (...) {                                                          \
        ::pic::set_error("%s: unexpected error", name);                    \
        return PIC_ERR_ARG;                                                \
    }

// device-memory hooks installed by pic_set_allocator (nulls: cudaMalloc / cudaFree)
struct Allocator {
    pic_alloc_fn alloc = nullptr;
    pic_free_fn free = nullptr;
    void *ctx = nullptr;
};
Allocator current_allocator();

// Tensor-core inference state of a surrogate network (k_mlp_tc.cu): BF16 weights of every
// member and layer, zero-padded to multiples of 16 and stored in the tensor core's
// no-swizzle K-major layout (8 x 8 core matrices, K-adjacent ones contiguous), and FP32
// biases.  Usable when every layer width is at most 256.
constexpr int MLP_MAX_LAYERS = 16;
struct MlpTc {
    int E = 0, L = 0;
    int k[MLP_MAX_LAYERS] = {}, n[MLP_MAX_LAYERS] = {};    // widths: in, out
    int kp[MLP_MAX_LAYERS] = {}, np[MLP_MAX_LAYERS] = {};  // padded to multiples of 16
    long long woff[MLP_MAX_LAYERS] = {}, boff[MLP_MAX_LAYERS] = {};
    long long wmember = 0, bmember = 0;                     // elements per member
    uint16_t *w = nullptr;                                  // E * wmember BF16
    float *b = nullptr;                                     // E * bmember
    unsigned int *err = nullptr;                            // bounded-wait timeouts
    long long wait_polls = 1LL << 22;                       // polls of a pipeline wait
    bool ok = false;
};
// FP32 parameters (per member: W_l (n x k), b_l at woff / boff, member stride P) -> tc
void mlp_tc_pack(const MlpTc &tc, const float *params, long long P, const long long *woff,
                 const long long *boff, cudaStream_t s);
// Y (E x n x outputs, FP32) from X (n x inputs, FP32); PIC_ERR_TIMEOUT if a wait gave up
pic_status mlp_tc_forward(const MlpTc &tc, const float *X, float *Y, int64_t n, cudaStream_t s);
// One product of the training path on the tensor cores, per member z of E:
// C(z)[m][n] (+)= sum_k A(z, m, k) B(z, k, n), operands FP32 addressed by strides (as the
// CUDA-core GEMM takes them), rounded to BF16 into the packed scratch buffers (A: E x
// roundup(M, 128) x roundup(K, 16), B: E x roundup(N, 16) x roundup(K, 16) elements), FP32
// accumulation in TMEM.  Needs N <= 256 and K <= 256 (false: not done).  Bounded waits
// that give up are counted in *err.
struct TcGemmOp {
    const float *A, *B;
    float *C;
    int M, N, K;
    long long sAz, sBz, sCz;
    int sAm, sAk, sBk, sBn, ldc;
    int accumulate;
};
bool mlp_tc_gemm(const TcGemmOp &g, int E, uint16_t *scratch_a, uint16_t *scratch_b,
                 unsigned int *err, cudaStream_t s);
#define PIC_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t err__ = (expr);                                                     \
        if (err__ != cudaSuccess) {                                                     \
            ::pic::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(err__), \
                             __FILE__, __LINE__);                                       \
            return PIC_ERR_CUDA;                                                        \
        }                                                                               \
    } while (0)

// ---------------------------------------------------------------------------------
// fixed point of the FP32 build
// ---------------------------------------------------------------------------------
// Barycentric coordinates are stored as integers in units of 2^-22 that sum to exactly
// 2^22.  The current of a segment, lambda_a^s lambda_b^e - lambda_b^s lambda_a^e, is then
// an exact integer in units of 2^-44 and node charges are integers in units of 2^-22:
// every scatter sum is exact and independent of summation order, and the discrete
// continuity equation holds identically in integers.
constexpr int LAM_BITS = 22;
constexpr int32_t LAM_ONE = 1 << LAM_BITS;
constexpr double LAM_INV = 1.0 / (double)LAM_ONE;
constexpr double J_INV = LAM_INV * LAM_INV;  // 2^-44

// ---------------------------------------------------------------------------------
// host mesh and operators
// ---------------------------------------------------------------------------------
struct HostMesh {
    pic_units units{};
    int64_t N0 = 0, N1 = 0, N2 = 0;
    std::vector<double> zr;            // N0 x 2 (z, rho)
    std::vector<int32_t> tri;          // N2 x 3, counter-clockwise in (z, rho)
    std::vector<int32_t> tri_edge;     // N2 x 3, local edge k opposite local node k
    std::vector<int32_t> tri_nbr;      // N2 x 3, neighbour across local edge k or -1
    std::vector<int32_t> edge_nodes;   // N1 x 2 (tail = lower index, head)
    std::vector<int32_t> edge_tag;     // N1: 0 interior or PIC_BC_*
    std::vector<int32_t> edge_face;    // N1 x 2 faces (or -1)
    std::vector<int8_t> edge_face_sign;// N1 x 2: D_curl entry of (face, edge)
    std::vector<double> area;          // N2
    std::vector<double> grad;          // N2 x 3 x 2: grad(lambda_k) (d/dz, d/drho)
    std::vector<double> mu_inv;        // N2: diagonal of star_mu^-1
    std::vector<int64_t> eps_ptr;      // star_eps in CSR, N1 rows
    std::vector<int32_t> eps_idx;
    std::vector<double> eps_val;
    std::vector<int32_t> free_edges;   // non-PEC edges, ascending
    std::vector<int32_t> free_of_edge; // N1: index in free_edges or -1
    std::vector<uint8_t> node_on_pec;  // N0
    bool have_spai = false;
    std::vector<int64_t> M_ptr;        // SPAI M in CSR over free edges
    std::vector<int32_t> M_idx;
    std::vector<double> M_val;
    double dt_stable = 0.0;
    double lambda_max = 0.0;
    // uniform bucket grid over triangle bounding boxes, for point location
    double bb_z0 = 0, bb_r0 = 0, bb_h = 1;
    int64_t bb_nz = 0, bb_nr = 0;
    std::vector<int64_t> bb_ptr;
    std::vector<int32_t> bb_tri;
};

// local edge k joins local nodes (k+1)%3 and (k+2)%3; its tail is the lower node index
inline void edge_tail_head(const int32_t *n3, int k, int *a, int *b) {
    int i = (k + 1) % 3, j = (k + 2) % 3;
    if (n3[i] < n3[j]) { *a = i; *b = j; } else { *a = j; *b = i; }
}

// run f(begin, end) over [0, n) on the host's cores
template <class F>
void parallel_for(int64_t n, F &&f) {
    unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    if (n < 4096 || nt == 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> th;
    int64_t chunk = (n + nt - 1) / nt;
    for (unsigned i = 0; i < nt; i++) {
        int64_t a = (int64_t)i * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        th.emplace_back([=, &f] { f(a, b); });
    }
    for (auto &t : th) t.join();
}

void build_locator(HostMesh &m);
// containing triangle (largest smallest barycentric coordinate) or -1; lam[3] out
int32_t locate_point(const HostMesh &m, double z, double rho, double lam[3]);
// intervals of the line z = z0, rho in [rho0, rho1], per triangle crossed (sorted, with
// the barycentric coordinates at both ends); false if the line leaves the mesh, passes
// through a node's z or the intervals do not tile [rho0, rho1]
bool build_emit_line(const HostMesh &m, double z0, double rho0, double rho1,
                     std::vector<double> &rho_a, std::vector<double> &rho_b,
                     std::vector<double> &lam_a, std::vector<double> &lam_b,
                     std::vector<int32_t> &tri);

// Kernels the library has enqueued for execution in this process.  Every launch site adds
// one; a stream capture runs nothing, so the kernels it recorded are taken back out and
// added again at each replay of the graph.
void note_launches(long long k);
long long launches_this_thread();
#define PIC_LAUNCHED() ::pic::note_launches(1)

// ---------------------------------------------------------------------------------
// device layouts
// ---------------------------------------------------------------------------------
// One record per triangle, read by the particle kernel: static geometry and topology,
// plus the per-step field coefficients written by the field kernel.  The E field inside
// the triangle is linear in lambda: E(lambda) = sum_k lambda_k c_k (components z, rho);
// bphi = (B^{n+1/2} + B^{n-1/2}) / (2 A) is the time-centred B_phi (W2 = 1/A).
template <class R>
struct alignas(sizeof(R) == 4 ? 128 : 64) TriRec {
    R g[4];       // grad lambda_0 (z, rho), grad lambda_1 (z, rho); grad lambda_2 = -g0 - g1
    R rho[3];     // node rho
    R inv_area;
    R c[6];       // c_0 (z, rho), c_1, c_2
    R bphi;
    R pad;
    int32_t node[3];
    int32_t flags; // bit k: local edge k runs (k+1)%3 -> (k+2)%3 (D_curl entry +1)
    int32_t edge[3];
    int32_t eflags; // = flags, beside the edges: one 16-byte load gives both
    int32_t nbr[3]; // neighbour triangle, or -(PIC_BC_* tag) on the boundary
    int32_t entry;  // bits 2k, 2k+1: local index, in nbr[k], of the node opposite the
                    // shared edge (the mesh is conforming and counter-clockwise, so the
                    // neighbour runs that edge the other way: its node entry+1 is this
                    // triangle's node k+2, its node entry+2 is node k+1)
};

struct PF32 {
    using R = float;
    using Lam = int32_t;
    using Acc = unsigned long long;  // two's-complement int64 accumulators
    static constexpr bool fixed = true;
};
struct PF64 {
    using R = double;
    using Lam = double;
    using Acc = double;
    static constexpr bool fixed = false;
};

template <class P>
struct Particles {
    int32_t *tri = nullptr;
    typename P::Lam *l0 = nullptr, *l1 = nullptr;
    typename P::R *ur = nullptr, *up = nullptr, *uz = nullptr;
    int32_t *pid = nullptr;
};

enum {
    CNT_ABSORBED = 0,
    CNT_OVERFLOW = 1,
    CNT_CROSSINGS = 2,
    CNT_REMAINDER = 3,  // nodes where D_div J was not a multiple of 2^22 (must stay 0)
    CNT_TIMEOUT = 4,    // bounded device waits that gave up (must stay 0)
    CNT_EMITTED = 5,    // particles born by the emitter
    CNT_NEXT_PID = 6,   // next particle id once an emitter was set
    CNT_EMIT_DROPPED = 7,   // particles the emitter did not make for lack of room
    CNT_N = 8
};
// slots past the capacity that the particle arrays keep for 16-byte bulk-copy rounding
constexpr int64_t SLOT_PAD = 8;

template <class P>
struct PushArgs {
    const TriRec<typename P::R> *rec;
    Particles<P> p;
    const int64_t *n_slots;     // device count of slots
    typename P::Acc *J;         // N1, units: fixed 2^-44 (FP32) / 1 (FP64) of q_src/dt
    typename P::Acc *Q;         // N0, Q^{n+1}, units 2^-22 / 1 of q_src
    typename P::Acc *Qabs;      // N0
    unsigned long long *counters;
    typename P::R qmdt2;        // q dt / (2 m)
    typename P::R dt;
    typename P::R inv_c2;
    typename P::R bz;
    int32_t walk_cap;
    int32_t ctas_per_sm;        // launch shape: persistent CTAs per SM (0: as many as fit)
    int32_t pusher;             // PIC_PUSHER_BORIS or PIC_PUSHER_VAY (Eq. DLE)
    int64_t wait_polls;         // FP32 kernel: polls before a tile-pipeline wait gives up
};
// default of PushArgs::wait_polls (each poll suspends the thread for at most 100 us)
constexpr int64_t PUSH_WAIT_POLLS = 1LL << 14;

// Emission line z = const, cut into the triangles it crosses: interval k spans
// rho in [rho_a[k], rho_b[k]] inside triangle tri[k], with barycentric coordinates lam_a
// and lam_b (3 each) at its ends (linear in between).
struct EmitLine {
    const double *rho_a, *rho_b, *lam_a, *lam_b;
    const int32_t *tri;
    int32_t n;
};

template <class P>
struct EmitArgs {
    EmitLine line;
    Particles<P> p;
    const TriRec<typename P::R> *rec;
    int64_t *n_slots;
    unsigned long long *counters;
    typename P::Acc *Qn;        // Q^n: the births' charge is added here
    typename P::Acc *Qwall;     // and taken out of the Gauss-law bookkeeping here
    int64_t cap, per_step;
    double rho0, rho1, u_normal, u_thermal;
    unsigned long long seed;
};

template <class P>
void launch_emit(const EmitArgs<P> &a, cudaStream_t s);

// field probes: group g owns entries [ptr[g], ptr[g+1]) of (face, weight); state[0] is
// the step phase, state[1] the records written, state[2] the records dropped
template <class P>
struct ProbeArgs {
    const typename P::R *B;
    const int64_t *ptr;
    const int32_t *face;
    const double *weight;
    const int32_t *power;
    double *buf;            // capacity x n_groups
    long long *state;
    unsigned *done;
    int32_t n_groups, every;
    long long capacity;
};

template <class P>
void launch_probe(const ProbeArgs<P> &a, cudaStream_t s);

// output ports: port k owns entries [ptr[k], ptr[k+1]) of (triangle, barycentric point,
// quadrature weight); after the face kernel of a step, P_k = sum w E_rho(lambda) B_phi
// from the triangle records (E^n and the time-centred B_phi); every `every` steps the
// ports' values are appended to a device buffer; state as for the probes
template <class P>
struct PortArgs {
    const TriRec<typename P::R> *rec;
    const int64_t *ptr;
    const int32_t *tri;
    const double *lam;      // 3 per entry
    const double *weight;
    double *buf;            // capacity x n_ports
    long long *state;
    unsigned *done;
    int32_t n_ports, every;
    long long capacity;
};

template <class P>
void launch_port(const PortArgs<P> &a, cudaStream_t s);

template <class P>
struct FieldArgs {
    TriRec<typename P::R> *rec;
    typename P::R *E;           // N1
    const typename P::R *Es;    // N1 static field added at the gather only, or null
    // lossy (absorbing) layer, or null: per free-edge row (a, b) with
    // E <- a E + b dt (M r), per face (a, b) with B <- a B - b dt (D_curl E)
    const typename P::R *loss_e;  // nf x 2
    const typename P::R *loss_f;  // N2 x 2
    typename P::R *B;           // N2, B^{n-1/2} in, B^{n+1/2} out
    const typename P::R *mu_inv;// N2
    const int32_t *edge_face;   // nf x 2, per free edge: (face+1) * sign, 0 if none
    const int32_t *free_edges;  // nf
    typename P::Acc *J;         // N1 (zeroed by the face kernel before the particle step)
    double *D;                  // N1 auxiliary dual flux (DGL)
    typename P::R *r;           // nf scratch: D_curl^T star_mu^-1 B - J
    // M in sliced ELL: slices of 32 rows, column-major inside a slice
    const int64_t *ell_off;     // n_slices + 1, element offset of each slice
    const int32_t *ell_col;
    const typename P::R *ell_val;
    int64_t N1, N2, nf;
    typename P::R dt;
    double j_scale;             // physical J = J_acc * j_scale
    // FP32 build: Q^{n+1} = Q^n - D_div J / 2^22 - Q_absorbed per node (exact)
    const int64_t *node_ptr;    // N0 + 1: node -> incident edges
    const int32_t *node_edge;
    const int8_t *node_sign;    // +1 tail, -1 head
    const typename P::Acc *Qn;
    typename P::Acc *Qabs;      // N0 (zeroed by the face kernel before the particle step)
    typename P::Acc *Qnext;
    typename P::Acc *Qwall;     // N0: charge removed at walls since the Gauss-law reference
    unsigned long long *counters;
    int64_t N0;
    int32_t block;              // launch shape: threads per block (<= 512)
};

template <class P> void launch_push(const PushArgs<P> &a, int64_t n_bound, cudaStream_t s);
void launch_push_f32(const PushArgs<PF32> &a, int64_t n_bound, cudaStream_t s);
template <class P> void launch_field_b(const FieldArgs<P> &a, cudaStream_t s);
template <class P> void launch_field_e(const FieldArgs<P> &a, cudaStream_t s);
template <class P>
void launch_deposit_q(const TriRec<typename P::R> *rec, Particles<P> p, int64_t first,
                      int64_t count, typename P::Acc *Q, cudaStream_t s);

struct SortScratch {
    int32_t *cnt = nullptr;      // N2 + 1: counts, then write cursors
    int32_t *blk = nullptr;      // scan chunk sums
    int64_t *n_old = nullptr;    // slot count before the sort
};
// stable-enough counting sort by triangle; drops removed particles; writes the new
// slot count to *n_slots (device)
template <class P>
void launch_resort(Particles<P> src, Particles<P> dst, int64_t *n_slots, int64_t n_bound,
                   int64_t N2, const SortScratch &sc, cudaStream_t s);

// diagnostics, FP64 reductions on the device
struct DiagDev {
    const int64_t *node_ptr;     // N0 + 1: node -> incident edges (CSR)
    const int32_t *node_edge;    // incident edge
    const int8_t *node_sign;     // D_div entry: +1 tail, -1 head
    const uint8_t *node_on_pec;  // N0
    const int64_t *eps_ptr;      // star_eps CSR
    const int32_t *eps_idx;
    const double *eps_val;
    int64_t N0, N1, N2;
};
// out[0]: max |dce| (units of q_src), out[1]: count of nonzero dce (fixed: exact),
// out[2]: max |NR_DCE|, out[3]: max |dgl - ref|, out[4]: max |Q|, out[5]: field energy,
// out[6]: sum (gamma - 1) over live particles
template <class P>
void launch_diag(const DiagDev &d, const typename P::Acc *J, const typename P::Acc *Qn,
                 const typename P::Acc *Qp, const typename P::Acc *Qabs,
                 const typename P::Acc *Qpos, const typename P::Acc *Qwall, const double *D,
                 double *dgl_ref, int set_ref, const typename P::R *E,
                 const typename P::R *B, const typename P::R *mu_inv, Particles<P> p,
                 const int64_t *n_slots, int64_t n_bound, double q_scale, double inv_c2,
                 double *out, cudaStream_t s);
template <class P>
void launch_export(Particles<P> p, int64_t n, const TriRec<typename P::R> *rec,
                   double *lam3, double *u3, int64_t *pid, cudaStream_t s);
template <class P>
void launch_acc_to_double(const typename P::Acc *a, double *out, int64_t n, double scale,
                          cudaStream_t s);

}  // namespace pic

struct pic_mesh {
    pic::HostMesh h;
};
