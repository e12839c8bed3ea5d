// K1, FP32 build: fused particle step -- Whitney gather, relativistic push (Boris, or the
// Vay form of Eq. DLE: one instantiation each), rotate-back to the meridian plane, triangle
// walk, charge-conserving current scatter.
//
// Positions are fixed-point barycentric coordinates (integers in units of 2^-22 that sum
// to 2^22).  Every segment's current lambda_a^s lambda_b^e - lambda_b^s lambda_a^e
// (Eq. current) is then an exact int64 and the scatter is exact and order-independent.
// Node charges are not scattered here: because the per-particle identity behind Eq. DCE
// holds exactly in these integers, Q^{n+1} = Q^n - D_div J / 2^22 - Q_absorbed is computed
// per node afterwards and equals Eq. charge bit for bit (the diagnostics recompute it
// from the positions and compare).
//
// Work split (persistent CTAs, warp-specialised):
//  * one producer warp (lane 0) stages tiles of TILE slots (structure of arrays, sorted
//    by triangle) into shared memory with 1-D bulk copies, STAGES buffers deep; a
//    buffer is refilled once all compute warps have arrived on its "empty" mbarrier;
//  * 8 compute warps advance two slots per thread per tile, branch-free: gather, push,
//    rotate-back and the end point in the start triangle.  For the ~4 in 5 particles
//    whose end point stays there, the edge currents are summed over the lanes that
//    share the triangle (match.any, then redux.sync on two 23-bit limbs) and one lane
//    per triangle issues the atomics.  A particle that leaves its triangle is appended,
//    with its start point and displacement, to its warp's ring in shared memory;
//  * whenever 32 entries are waiting, the warp walks them with all lanes: per triangle
//    the segment to the first edge reached, its currents (direct atomics), then the
//    neighbour (entered through a precomputed local edge index) until the end point,
//    the axis, a wall or the walk cap.  The remainder (< 32) is walked at the end.
// Every wait is bounded: on timeout the error counter is set and the CTA leaves once the
// producer lane has waited (bounded) for every bulk copy it issued.  Small arrays are indexed statically
// (nothing in local memory); fixed <-> float conversions use exact magic-number
// arithmetic instead of the quarter-rate converters.
#include <algorithm>

#include "pic_internal.h"

namespace pic {

namespace {

constexpr float INV = (float)LAM_INV;
constexpr float ONEF = (float)LAM_ONE;
constexpr float TWO23 = 8388608.0f;
constexpr int TWO23_BITS = 0x4B000000;

constexpr int CW = 8;              // compute warps per CTA
constexpr int PT = CW * 32;        // compute threads per CTA
constexpr int NT = PT + 32;        // plus one producer warp
constexpr int ROUNDS = 2;          // slots per compute thread per tile
constexpr int TILE = PT * ROUNDS;  // slots per tile
constexpr int STAGES = 2;          // tile buffers in flight
constexpr int QCAP = 64;           // ring entries per compute warp (at most 31 + 32 used)
constexpr unsigned WAIT_SLICE_NS = 100000;    // one bounded mbarrier poll sleeps <= 100 us
constexpr long long WAIT_LIMIT = PUSH_WAIT_POLLS;   // polls of a drain wait (<= ~1.6 s)

// s in [0, 2^23): exactly (float)s * 2^-22
__device__ __forceinline__ float fix2f(int s) {
    return (__int_as_float(s | TWO23_BITS) - TWO23) * INV;
}
// x in [0, 2): round-to-nearest of x * 2^22 (the FMA rounds x 2^22 + 2^23 once)
__device__ __forceinline__ int f2fix(float x) {
    return __float_as_int(fmaf(x, ONEF, TWO23)) - TWO23_BITS;
}

__device__ __forceinline__ const float4 *rec4(const TriRec<float> *rec, int t) {
    return reinterpret_cast<const float4 *>(rec + t);
}
__device__ __forceinline__ const int4 *rec4i(const TriRec<float> *rec, int t) {
    return reinterpret_cast<const int4 *>(rec + t);
}

__device__ __forceinline__ void red_add(unsigned long long *p, long long v) {
    atomicAdd(p, (unsigned long long)v);
}

// Sum a signed value |v| < 2^45 over the lanes of grp: redux.sync on the two 23-bit limbs
// of v + 2^45 (each limb sum stays below 2^28).
__device__ __forceinline__ long long group_sum(unsigned grp, int n, long long v) {
    const long long bias = 1LL << 45;
    unsigned long long b = (unsigned long long)(v + bias);
    unsigned slo = __reduce_add_sync(grp, (unsigned)(b & 0x7FFFFFu));
    unsigned shi = __reduce_add_sync(grp, (unsigned)(b >> 23));
    return ((long long)shi << 23) + (long long)slo - (long long)n * bias;
}

__device__ __forceinline__ int sel3(int k, int a, int b, int c) { return k == 0 ? a : (k == 1 ? b : c); }
__device__ __forceinline__ float self3(int k, float a, float b, float c) {
    return k == 0 ? a : (k == 1 ? b : c);
}

// The floating-point steps of the walk are spelled out with explicit rounding: the walk is
// inlined at more than one call site, and a particle must get the same bits whichever site
// (ring pass or final flush) handles it, so that runs are reproducible whatever order a
// re-sort leaves the particles of one triangle in.
// barycentric image of a meridian displacement: g_z d0 + g_rho d1
__device__ __forceinline__ float bary_step(float gz, float gr, float d0, float d1) {
    return __fmaf_rn(gz, d0, __fmul_rn(gr, d1));
}

struct Seg {
    int e0, e1, e2;  // end point (fixed point)
    int kx;          // exit edge, or -1 when the segment ends inside the triangle
    float sx;        // fraction of the remaining displacement used
};

// End of the segment that starts at f (float of the fixed-point start) and moves by dl,
// in one triangle.  The exit edge is the one reached first (smallest parameter, ties to
// the lower index), never the edge just entered; the crossing point has coordinate kx
// exactly 0 and the other two summing to 2^22.
__device__ __forceinline__ Seg segment_end(float f0, float f1, float f2, float dl0, float dl1,
                                           float dl2, int entered) {
    Seg r;
    const float le0 = f0 + dl0, le1 = f1 + dl1, le2 = f2 + dl2;
    const bool x0 = le0 < 0.f && entered != 0;
    const bool x1 = le1 < 0.f && entered != 1;
    const bool x2 = le2 < 0.f && entered != 2;
    if (!(x0 || x1 || x2)) {
        r.kx = -1;
        r.sx = 1.f;
        r.e0 = f2fix(fmaxf(le0, 0.f));
        r.e1 = f2fix(fmaxf(le1, 0.f));
        r.e2 = LAM_ONE - r.e0 - r.e1;
        if (r.e2 < 0) {
            if (r.e0 >= r.e1) r.e0 += r.e2; else r.e1 += r.e2;
            r.e2 = 0;
        }
        return r;
    }
    const float sA = x0 ? __fdividef(f0, f0 - le0) : 2.f;
    const float sB = x1 ? __fdividef(f1, f1 - le1) : 2.f;
    const float sC = x2 ? __fdividef(f2, f2 - le2) : 2.f;
    if (sA <= sB && sA <= sC) { r.kx = 0; r.sx = sA; }
    else if (sB <= sC) { r.kx = 1; r.sx = sB; }
    else { r.kx = 2; r.sx = sC; }
    const int kx = r.kx;
    const float ci = fmaxf(__fmaf_rn(r.sx, self3(kx, dl1, dl2, dl0), self3(kx, f1, f2, f0)), 0.f);
    const float cj = fmaxf(__fmaf_rn(r.sx, self3(kx, dl2, dl0, dl1), self3(kx, f2, f0, f1)), 0.f);
    int qi = f2fix(fminf(__fdividef(ci, ci + cj), 1.f));
    qi = min(max(qi, 0), LAM_ONE);
    const int qj = LAM_ONE - qi;
    r.e0 = kx == 0 ? 0 : (kx == 1 ? qj : qi);
    r.e1 = kx == 1 ? 0 : (kx == 2 ? qj : qi);
    r.e2 = kx == 2 ? 0 : (kx == 0 ? qj : qi);
    return r;
}

// Eq. current of a segment s -> e inside one triangle.  With the local edges oriented
// counter-clockwise (edge 0: 1->2, 1: 2->0, 2: 0->1) the currents are
//   A0 = s1 e2 - s2 e1,  A1 = s2 e0 - s0 e2,  A2 = s0 e1 - s1 e0,
// and because s and e both sum to 2^22, the net outflow at each node is
//   A2 - A1 = 2^22 (s0 - e0),  A0 - A2 = 2^22 (s1 - e1)   (the identity behind Eq. DCE).
// So one 64-bit product pair (A1) and two 32-bit differences determine all three, also
// after summing over particles of the same triangle.
__device__ __forceinline__ void ccw_from(long long A1, int d0, int d1, long long &A0,
                                         long long &A2) {
    A2 = A1 + ((long long)d0 << LAM_BITS);
    A0 = A2 + ((long long)d1 << LAM_BITS);
}
// the ccw currents with the global orientation of each edge applied (flags bit k: local
// edge k runs (k+1)%3 -> (k+2)%3, i.e. from its lower to its higher node index)
__device__ __forceinline__ void oriented(int flags, long long &A0, long long &A1, long long &A2) {
    if (!(flags & 1)) A0 = -A0;
    if (!(flags & 2)) A1 = -A1;
    if (!(flags & 4)) A2 = -A2;
}

// the three oriented currents of one segment s -> e
__device__ __forceinline__ void currents(int s0, int s1, int s2, const Seg &e, int flags,
                                         long long &J0, long long &J1, long long &J2) {
    J1 = (long long)s2 * e.e0 - (long long)s0 * e.e2;
    ccw_from(J1, s0 - e.e0, s1 - e.e1, J0, J2);
    oriented(flags, J0, J1, J2);
}

// a particle whose displacement leaves its start triangle t: slot, start point (s0, s1,
// 2^22 - s0 - s1), meridian displacement (d0, d1) and its image (dl0, dl1) in t's
// barycentric coordinates
struct __align__(16) QEntry {
    int slot, t, s0, s1;
    float d0, d1, dl0, dl1;
};

// one tile of the structure-of-arrays particle state, staged by bulk copies
struct __align__(128) TileBuf {
    int tri[TILE];
    int l0[TILE];
    int l1[TILE];
    float ur[TILE];
    float up[TILE];
    float uz[TILE];
};

struct PushSmem {
    TileBuf buf[STAGES];
    QEntry q[CW][QCAP];                // per compute warp: ring of particles to walk on
    unsigned long long full[STAGES];   // the bulk copies of a stage's tile landed
    unsigned long long empty[STAGES];  // every compute warp released the stage
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes) : "memory");
}
// test for the phase; a waiting thread is suspended until the phase completes or the
// suspend-time hint (ns) runs out, instead of spinning
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(b)), "r"(parity), "n"(WAIT_SLICE_NS) : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; false when `polls` polls did not see it
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity,
                                          long long polls = WAIT_LIMIT) {
    for (long long k = 0; k < polls; k++)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
// 1-D bulk copy global -> shared, completing on the mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}
// producer lane: stage tile `tile` (slots [tile*TILE, tile*TILE + TILE) clipped to n, rounded up
// to 4 slots so every copy is a multiple of 16 bytes; the arrays have that much room)
__device__ __forceinline__ void issue_tile(const PushArgs<PF32> &a, PushSmem &sm, int stage,
                                           long long tile, long long n) {
    const long long base = tile * TILE;
    const long long cnt = min((long long)TILE, n - base);
    const unsigned bytes = (unsigned)(((cnt + 3) & ~3LL) * 4);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    unsigned long long *bar = &sm.full[stage];
    mbar_expect_tx(bar, 6 * bytes);
    TileBuf &b = sm.buf[stage];
    bulk_load(b.tri, a.p.tri + base, bytes, bar);
    bulk_load(b.l0, a.p.l0 + base, bytes, bar);
    bulk_load(b.l1, a.p.l1 + base, bytes, bar);
    bulk_load(b.ur, a.p.ur + base, bytes, bar);
    bulk_load(b.up, a.p.up + base, bytes, bar);
    bulk_load(b.uz, a.p.uz + base, bytes, bar);
}

// Gather, push, rotate-back and the end of the move for one particle (slot i, state from
// the staged tile).  A particle whose end point stays in its start triangle t0 gets its
// current as (A1, s0 - e0, s1 - e1) (see ccw_from) and its new position stored; one that
// leaves t0 is described in e, flagged, and contributes no current here (its whole path,
// the part in t0 included, is walked later).
template <bool VAY>
__device__ __forceinline__ void push_particle(const PushArgs<PF32> &a, int i, int t0, int s0,
                                              int s1, float ur, float up, float uz,
                                              long long &a1, int &dq0, int &dq1, int4 &EG,
                                              bool &crossed, QEntry &e) {
    const float4 *R = rec4(a.rec, t0);
    const float4 G = __ldg(R + 0), RH = __ldg(R + 1), CA = __ldg(R + 2), CB = __ldg(R + 3);
    EG = __ldg(rec4i(a.rec, t0) + 5);   // edges and orientation flags
    const int s2 = LAM_ONE - s0 - s1;
    const float f0 = fix2f(s0), f1 = fix2f(s1), f2 = fix2f(s2);

    // gather (Sec. 3.2): E(lambda) = sum_k lambda_k c_k, time-centred B_phi, guide B_z
    const float Ez = f0 * CA.x + f1 * CA.z + f2 * CB.x;
    const float Er = f0 * CA.y + f1 * CA.w + f2 * CB.y;
    const float rho = f0 * RH.x + f1 * RH.y + f2 * RH.z;
    const float h = a.qmdt2;

    if constexpr (VAY) {
        // Eq. DLE with the mean of v^{n-1/2} and v^{n+1/2} in the magnetic term (Vay),
        // solved in closed form: u' = u + 2h E + h (u / gamma) x B, tau = h B, gamma_new^2
        // the positive root of g^4 - sigma g^2 - (tau^2 + (u'.tau)^2 / c^2),
        // t = tau / gamma_new, u = (u' + (u'.t) t + u' x t) / (1 + t^2)
        const float gi = rsqrtf(1.f + (ur * ur + up * up + uz * uz) * a.inv_c2);
        const float tp = h * CB.z, tz = h * a.bz;
        const float pr = ur + 2.f * h * Er + gi * (up * tz - uz * tp);
        const float pp = up - gi * ur * tz;
        const float pz = uz + 2.f * h * Ez + gi * ur * tp;
        const float tau2 = tp * tp + tz * tz;
        const float ut0 = pp * tp + pz * tz;
        const float x = tau2 + ut0 * ut0 * a.inv_c2;
        const float sigma = 1.f + (pr * pr + pp * pp + pz * pz) * a.inv_c2 - tau2;
        const float disc = sqrtf(sigma * sigma + 4.f * x);
        const float g2 = sigma >= 0.f ? 0.5f * (sigma + disc) : __fdividef(2.f * x, disc - sigma);
        const float gn = rsqrtf(g2);
        const float qp = tp * gn, qz = tz * gn;
        const float ut = pp * qp + pz * qz;
        const float sf = __fdividef(1.f, 1.f + qp * qp + qz * qz);
        ur = sf * (pr + pp * qz - pz * qp);
        up = sf * (pp + ut * qp - pr * qz);
        uz = sf * (pz + ut * qz + pr * qp);
    } else {
        // relativistic Boris (Eq. DLE): half kick, rotation about B = (0, B_phi, B_z), half
        // kick
        ur += h * Er;
        uz += h * Ez;
        const float gi = rsqrtf(1.f + (ur * ur + up * up + uz * uz) * a.inv_c2);
        const float tp = h * CB.z * gi, tz = h * a.bz * gi;
        const float sf = __fdividef(2.f, 1.f + tp * tp + tz * tz);
        const float pr = ur + (up * tz - uz * tp);   // u' = u- + u- x t, t = (0, tp, tz)
        const float pp = up - ur * tz;
        const float pz = uz + ur * tp;
        ur += sf * (pp * tz - pz * tp) + h * Er;      // u+ = u- + u' x (sf t), then half kick
        up -= sf * pr * tz;
        uz += sf * pr * tp + h * Ez;
    }

    // move (Eq. DNE) in the ring's Cartesian frame, rotate back to the meridian plane
    const float gi = rsqrtf(1.f + (ur * ur + up * up + uz * uz) * a.inv_c2);
    const float xr = ur * gi * a.dt, yp = up * gi * a.dt;
    const float x = rho + xr;
    const float rn2 = x * x + yp * yp;
    const float d0 = uz * gi * a.dt;
    float d1 = 0.f;
    if (rn2 > 0.f) {
        const float rinv = rsqrtf(rn2);
        d1 = __fdividef(2.f * rho * xr + xr * xr + yp * yp, rn2 * rinv + rho);
        const float cs = x * rinv, sn = yp * rinv;
        const float nr = cs * ur + sn * up;
        up = -sn * ur + cs * up;
        ur = nr;
    }
    __stcs(a.p.ur + i, ur);
    __stcs(a.p.up + i, up);
    __stcs(a.p.uz + i, uz);

    // end point in barycentric coordinates of t0
    const float dl0 = bary_step(G.x, G.y, d0, d1), dl1 = bary_step(G.z, G.w, d0, d1);
    const float le0 = f0 + dl0, le1 = f1 + dl1, le2 = f2 - (dl0 + dl1);
    crossed = !(le0 >= 0.f && le1 >= 0.f && le2 >= 0.f);
    // inside t0: round to fixed point summing to 2^22 (a rounding deficit of the remainder
    // goes to the larger of the other two coordinates).  A particle that leaves keeps
    // e = s here, i.e. zero current.
    int e0 = f2fix(le0), e1 = f2fix(le1);
    int e2 = LAM_ONE - e0 - e1;
    const int neg = min(e2, 0);
    const bool big0 = e0 >= e1;
    e0 += big0 ? neg : 0;
    e1 += big0 ? 0 : neg;
    e2 -= neg;
    if (crossed) {
        e0 = s0;
        e1 = s1;
        e2 = s2;
    }
    a1 = (long long)s2 * e0 - (long long)s0 * e2;
    dq0 = s0 - e0;
    dq1 = s1 - e1;
    if (!crossed) {
        __stcs(a.p.l0 + i, e0);
        __stcs(a.p.l1 + i, e1);
    }
    e = QEntry{i, t0, s0, s1, d0, d1, dl0, dl1};
}

__device__ __forceinline__ void store_position(const PushArgs<PF32> &a, int slot, int t, int e0,
                                               int e1) {
    __stcs(a.p.tri + slot, t);
    __stcs(a.p.l0 + slot, e0);
    __stcs(a.p.l1 + slot, e1);
}

// Walk the particles of one ring pass (all 32 lanes call this; lanes with valid = false
// only take part in the warp-wide steps).  Per triangle: the segment to the end point or
// to the first edge reached, its Eq. current, then the neighbour across that edge, where
// the two shared nodes keep their coordinates.  The first segments lie in the triangles
// the particles started in, which the lanes of a pass mostly share: their currents are
// summed per triangle like those of the particles that stay; later segments deposit with
// direct atomics.  The walk stops on the axis (the meridian segment stays at rho >= 0)
// and removes the particle at a wall or at the walk cap (its charge goes to Q_abs).
// Returns the number of edges reached.
__device__ __forceinline__ unsigned walk_pass(const PushArgs<PF32> &a, const QEntry q, bool valid,
                                              int lane) {
    const unsigned full = 0xffffffffu;
    int t = valid ? q.t : -1;
    int s0 = q.s0, s1 = q.s1, s2 = LAM_ONE - q.s0 - q.s1;
    int4 EG = make_int4(0, 0, 0, 0), NB = EG;
    Seg sg{};
    long long a1 = 0;
    int dq0 = 0, dq1 = 0;
    if (valid) {
        EG = __ldg(rec4i(a.rec, t) + 5);   // edges, orientation flags
        NB = __ldg(rec4i(a.rec, t) + 6);   // neighbours, entry indices
        sg = segment_end(fix2f(s0), fix2f(s1), fix2f(s2), q.dl0, q.dl1, -(q.dl0 + q.dl1), -1);
        a1 = (long long)s2 * sg.e0 - (long long)s0 * sg.e2;
        dq0 = s0 - sg.e0;
        dq1 = s1 - sg.e1;
    }
    const unsigned grp = __match_any_sync(full, t);
    if (!valid) return 0;
    {
        const int cnt = __popc(grp);
        long long S1 = group_sum(grp, cnt, a1);
        const int D0 = (int)__reduce_add_sync(grp, (unsigned)dq0);
        const int D1 = (int)__reduce_add_sync(grp, (unsigned)dq1);
        if (lane == __ffs(grp) - 1) {
            long long S0, S2;
            ccw_from(S1, D0, D1, S0, S2);
            oriented(EG.w, S0, S1, S2);
            red_add(a.J + EG.x, S0);
            red_add(a.J + EG.y, S1);
            red_add(a.J + EG.z, S2);
        }
    }
    float d0 = q.d0, d1 = q.d1;
    for (int ncross = 0;; ncross++) {
        if (sg.kx < 0) {
            store_position(a, q.slot, t, sg.e0, sg.e1);
            return (unsigned)ncross;
        }
        const int kx = sg.kx;
        const int nb = sel3(kx, NB.x, NB.y, NB.z);
        if (nb < 0 && -nb == PIC_BC_AXIS) {
            store_position(a, q.slot, t, sg.e0, sg.e1);
            return (unsigned)ncross + 1;
        }
        if (nb < 0 || ncross + 1 >= a.walk_cap) {
            const int4 nd = __ldg(rec4i(a.rec, t) + 4);
            red_add(a.Qabs + nd.x, sg.e0);
            red_add(a.Qabs + nd.y, sg.e1);
            red_add(a.Qabs + nd.z, sg.e2);
            if (nb >= 0) atomicAdd(a.counters + CNT_OVERFLOW, 1ULL);
            atomicAdd(a.counters + CNT_ABSORBED, 1ULL);
            __stcs(a.p.tri + q.slot, -1);
            return (unsigned)ncross + 1;
        }
        // enter nb through its local edge j (opposite its node j): its node j+2 is node kx+1
        // of t, its node j+1 is node kx+2
        const int j = (NB.w >> (2 * kx)) & 3;
        const int ea = sel3(kx, sg.e1, sg.e2, sg.e0);
        const int eb = sel3(kx, sg.e2, sg.e0, sg.e1);
        s0 = j == 0 ? 0 : (j == 1 ? ea : eb);
        s1 = j == 1 ? 0 : (j == 2 ? ea : eb);
        s2 = j == 2 ? 0 : (j == 0 ? ea : eb);
        const float rest = 1.f - sg.sx;
        d0 = __fmul_rn(d0, rest);
        d1 = __fmul_rn(d1, rest);
        t = nb;
        const float4 G = __ldg(rec4(a.rec, t));
        EG = __ldg(rec4i(a.rec, t) + 5);
        NB = __ldg(rec4i(a.rec, t) + 6);
        const float dl0 = bary_step(G.x, G.y, d0, d1), dl1 = bary_step(G.z, G.w, d0, d1);
        sg = segment_end(fix2f(s0), fix2f(s1), fix2f(s2), dl0, dl1, -(dl0 + dl1), j);
        long long J0, J1, J2;
        currents(s0, s1, s2, sg, EG.w, J0, J1, J2);
        red_add(a.J + EG.x, J0);
        red_add(a.J + EG.y, J1);
        red_add(a.J + EG.z, J2);
    }
}

}  // namespace

template <bool VAY>
__global__ void __launch_bounds__(NT, 4) k_push_f32(PushArgs<PF32> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PushSmem &sm = *reinterpret_cast<PushSmem *>(smem_raw);
    const long long n = *a.n_slots;
    const long long ntiles = (n + TILE - 1) / TILE;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned full = 0xffffffffu;
    // each CTA takes a contiguous range of tiles: consecutive tiles hold neighbouring
    // triangles (slots are sorted by triangle), so their records stay in this SM's L1
    const long long per = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long tile0 = (long long)blockIdx.x * per, tile1 = min(ntiles, tile0 + per);
    if (tile0 >= tile1) return;
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], CW);
        }
        mbar_fence_init();
    }
    __syncthreads();
    unsigned cx = 0;

    if (warp == CW) {
        // ---- producer warp: lane 0 stages the CTA's tiles; a stage is refilled once every
        // compute warp has released its previous tile
        if (lane == 0) {
            long long it = 0;
            for (long long tile = tile0; tile < tile1; tile++, it++) {
                const int stage = (int)(it % STAGES);
                if (it >= STAGES &&
                    !mbar_wait(&sm.empty[stage], (unsigned)((it / STAGES - 1) & 1), a.wait_polls)) {
                    atomicAdd(a.counters + CNT_TIMEOUT, 1ULL);
                    break;
                }
                issue_tile(a, sm, stage, tile, n);
            }
            // before the block can exit, every copy issued into its shared memory has
            // landed: wait (bounded) for the last phase issued on each stage.  After a
            // normal run the compute warps have seen these phases and the waits return at
            // once; after a timeout they may not have.
            for (long long k = it > STAGES ? it - STAGES : 0; k < it; k++)
                if (!mbar_wait(&sm.full[(int)(k % STAGES)], (unsigned)((k / STAGES) & 1)))
                    atomicAdd(a.counters + CNT_TIMEOUT, 1ULL);
        }
    } else {
        // ---- compute warps.  Particles that leave their start triangle go to the warp's
        // own ring; whenever 32 are waiting the warp walks them with all lanes.
        QEntry *ring = sm.q[warp];
        const unsigned below = (1u << lane) - 1;
        unsigned head = 0, tail = 0;   // warp-uniform, ring index = value & (QCAP - 1)
        long long it = 0;
        for (long long tile = tile0; tile < tile1; tile++, it++) {
            const int stage = (int)(it % STAGES);
            const bool ok = mbar_wait(&sm.full[stage], (unsigned)((it / STAGES) & 1), a.wait_polls);
            if (__any_sync(full, !ok)) {
                // leave; the producer drains the copies in flight before the block exits
                if (lane == 0) atomicAdd(a.counters + CNT_TIMEOUT, 1ULL);
                break;
            }
            const TileBuf &b = sm.buf[stage];
            const long long base = tile * TILE;
            for (int r = 0; r < ROUNDS; r++) {
                const int k = r * PT + tid;
                const long long i = base + k;
                const int t0 = i < n ? b.tri[k] : -1;
                long long a1 = 0;
                int dq0 = 0, dq1 = 0;
                int4 EG = make_int4(0, 0, 0, 0);
                bool crossed = false;
                QEntry e;
                if (t0 >= 0)
                    push_particle<VAY>(a, (int)i, t0, b.l0[k], b.l1[k], b.ur[k], b.up[k], b.uz[k],
                                       a1, dq0, dq1, EG, crossed, e);
                // currents of the particles that stay: summed over the lanes of each start
                // triangle (one 64-bit and two 32-bit sums determine all three edges), one
                // set of atomics per triangle
                const unsigned grp = __match_any_sync(full, t0);
                if (t0 >= 0) {
                    const int cnt = __popc(grp);
                    long long S1 = group_sum(grp, cnt, a1);
                    const int D0 = (int)__reduce_add_sync(grp, (unsigned)dq0);
                    const int D1 = (int)__reduce_add_sync(grp, (unsigned)dq1);
                    if (lane == __ffs(grp) - 1) {
                        long long S0, S2;
                        ccw_from(S1, D0, D1, S0, S2);
                        oriented(EG.w, S0, S1, S2);
                        red_add(a.J + EG.x, S0);
                        red_add(a.J + EG.y, S1);
                        red_add(a.J + EG.z, S2);
                    }
                }
                // particles that leave go to this warp's ring (at most 31 + 32 entries)
                const unsigned qmask = __ballot_sync(full, crossed);
                if (crossed) ring[(tail + __popc(qmask & below)) & (QCAP - 1)] = e;
                tail += __popc(qmask);
                if (tail - head >= 32) {
                    __syncwarp();
                    cx += walk_pass(a, ring[(head + lane) & (QCAP - 1)], true, lane);
                    head += 32;
                    __syncwarp();
                }
            }
            // this warp is done reading the stage: release it to the producer
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.empty[stage]);
        }
        // the rest of the ring (fewer than 32 entries)
        __syncwarp();
        cx += walk_pass(a, ring[(head + lane) & (QCAP - 1)], lane < (int)(tail - head), lane);
    }
    const unsigned sx = __reduce_add_sync(full, cx);
    if (lane == 0 && sx) atomicAdd(a.counters + CNT_CROSSINGS, (unsigned long long)sx);
}

struct LaunchShape {
    int bps = 0, sms = 0;
};
static LaunchShape g_push_shape[2][64];

template <bool VAY>
static void launch_push_f32_as(const PushArgs<PF32> &a, int64_t n_bound, cudaStream_t s) {
    const int smem = (int)sizeof(PushSmem);
    int dev = 0;
    cudaGetDevice(&dev);
    LaunchShape &ps = g_push_shape[VAY ? 1 : 0][dev & 63];
    if (ps.bps == 0) {
        cudaFuncSetAttribute(k_push_f32<VAY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int bps = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_push_f32<VAY>, NT, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ps.bps = bps > 0 ? bps : 1;
        ps.sms = sms > 0 ? sms : 1;
    }
    const int64_t tiles = (n_bound + TILE - 1) / TILE;
    const int bps = a.ctas_per_sm > 0 ? std::min(a.ctas_per_sm, ps.bps) : ps.bps;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)ps.sms * bps);
    k_push_f32<VAY><<<(unsigned)grid, NT, smem, s>>>(a);
    PIC_LAUNCHED();
}

void launch_push_f32(const PushArgs<PF32> &a, int64_t n_bound, cudaStream_t s) {
    if (n_bound <= 0) return;
    if (a.pusher == PIC_PUSHER_VAY) launch_push_f32_as<true>(a, n_bound, s);
    else launch_push_f32_as<false>(a, n_bound, s);
}

}  // namespace pic
