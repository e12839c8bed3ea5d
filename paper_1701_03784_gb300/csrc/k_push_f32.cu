// K1, FP32 build: fused particle step -- Whitney gather, relativistic Boris push,
// rotate-back to the meridian plane, triangle walk, charge-conserving current scatter.
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
//  * thread 0 stages tiles of TILE slots (structure of arrays, sorted by triangle) into
//    shared memory with 1-D bulk copies on an mbarrier, double-buffered;
//  * 8 compute warps advance two slots per thread per tile: gather, Boris, rotate-back
//    and the first segment of the walk (the whole path for most particles).  The first
//    segment's edge currents are summed over the lanes that share a start triangle
//    (match.any, then redux.sync on two 23-bit limbs) and one lane per triangle issues
//    the atomics.  A particle whose first segment reaches an edge is put in the tile's
//    crossing queue in shared memory;
//  * 1 walker warp finishes the queued particles of tile k (boundary, neighbour entry,
//    further segments with direct atomics) while the compute warps work on tile k+1.
//    The two queue buffers are handed over with full/empty mbarriers.
// Every wait is bounded: on timeout the error counter is set and the CTA leaves after a
// bounded wait for its own bulk copy in flight.  Small arrays are indexed statically
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
constexpr int NT = PT + 32;        // plus one walker warp
constexpr int ROUNDS = 2;          // slots per compute thread per tile
constexpr int TILE = PT * ROUNDS;  // slots per tile
constexpr long long WAIT_LIMIT = 1LL << 20;  // bounded mbarrier polling

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
    if (v != 0) atomicAdd(p, (unsigned long long)v);
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
    const float ci = fmaxf(self3(kx, f1, f2, f0) + r.sx * self3(kx, dl1, dl2, dl0), 0.f);
    const float cj = fmaxf(self3(kx, f2, f0, f1) + r.sx * self3(kx, dl2, dl0, dl1), 0.f);
    int qi = f2fix(fminf(__fdividef(ci, ci + cj), 1.f));
    qi = min(max(qi, 0), LAM_ONE);
    const int qj = LAM_ONE - qi;
    r.e0 = kx == 0 ? 0 : (kx == 1 ? qj : qi);
    r.e1 = kx == 1 ? 0 : (kx == 2 ? qj : qi);
    r.e2 = kx == 2 ? 0 : (kx == 0 ? qj : qi);
    return r;
}

// Eq. current of the segment s -> e on the three local edges, each oriented from its lower
// to its higher node index (flags bit k: local edge k runs (k+1)%3 -> (k+2)%3)
__device__ __forceinline__ void currents(int s0, int s1, int s2, const Seg &e, int flags,
                                         long long &J0, long long &J1, long long &J2) {
    J0 = (long long)s1 * e.e2 - (long long)s2 * e.e1;
    J1 = (long long)s2 * e.e0 - (long long)s0 * e.e2;
    J2 = (long long)s0 * e.e1 - (long long)s1 * e.e0;
    if (!(flags & 1)) J0 = -J0;
    if (!(flags & 2)) J1 = -J1;
    if (!(flags & 4)) J2 = -J2;
}

// a particle that reached edge kx of triangle t at the fixed-point point (s0, s1, 2^22 -
// s0 - s1) and still moves by (d0, d1)
struct QEntry {
    int slot, t, kx, s0, s1;
    float d0, d1;
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
    TileBuf buf[2];
    QEntry q[2][TILE];
    unsigned long long tile_full[2];   // bulk copies of a tile landed
    unsigned long long q_full[2];      // the compute warps filled a queue buffer
    unsigned long long q_empty[2];     // the walker drained it
    int qn[2];
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
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; false when the limit is reached
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity) {
    for (long long k = 0; k < WAIT_LIMIT; k++)
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
// barrier of the compute warps only (named barrier 1), OR-reducing a flag
__device__ __forceinline__ bool compute_sync_or(bool v) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, 1, %2, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r) : "r"((unsigned)v), "n"(PT) : "memory");
    return r != 0;
}

// thread 0: stage tile `tile` (slots [tile*TILE, tile*TILE + TILE) clipped to n, rounded up
// to 4 slots so every copy is a multiple of 16 bytes; the arrays have that much room)
__device__ __forceinline__ void issue_tile(const PushArgs<PF32> &a, PushSmem &sm, int stage,
                                           long long tile, long long n) {
    const long long base = tile * TILE;
    const long long cnt = min((long long)TILE, n - base);
    const unsigned bytes = (unsigned)(((cnt + 3) & ~3LL) * 4);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    unsigned long long *bar = &sm.tile_full[stage];
    mbar_expect_tx(bar, 6 * bytes);
    TileBuf &b = sm.buf[stage];
    bulk_load(b.tri, a.p.tri + base, bytes, bar);
    bulk_load(b.l0, a.p.l0 + base, bytes, bar);
    bulk_load(b.l1, a.p.l1 + base, bytes, bar);
    bulk_load(b.ur, a.p.ur + base, bytes, bar);
    bulk_load(b.up, a.p.up + base, bytes, bar);
    bulk_load(b.uz, a.p.uz + base, bytes, bar);
}

// Gather, Boris, rotate-back and the first segment of one particle (slot i, state from the
// staged tile).  Returns the first segment's three edge currents; a particle whose
// segment reaches an edge is described in e and flagged.
__device__ __forceinline__ void push_first(const PushArgs<PF32> &a, int i, int t0, int s0,
                                           int s1, float ur, float up, float uz, long long &j0a,
                                           long long &j0b, long long &j0c, bool &crossed,
                                           QEntry &e) {
    const float4 *R = rec4(a.rec, t0);
    const float4 G = __ldg(R + 0), RH = __ldg(R + 1), CA = __ldg(R + 2), CB = __ldg(R + 3);
    const int flags = __ldg(&reinterpret_cast<const int *>(a.rec + t0)[4 * 4 + 3]);
    const int s2 = LAM_ONE - s0 - s1;
    const float f0 = fix2f(s0), f1 = fix2f(s1), f2 = fix2f(s2);

    // gather (Sec. 3.2): E(lambda) = sum_k lambda_k c_k, time-centred B_phi, guide B_z
    const float Ez = f0 * CA.x + f1 * CA.z + f2 * CB.x;
    const float Er = f0 * CA.y + f1 * CA.w + f2 * CB.y;
    const float rho = f0 * RH.x + f1 * RH.y + f2 * RH.z;
    const float h = a.qmdt2;

    // relativistic Boris (Eq. DLE): half kick, rotation about B = (0, B_phi, B_z), half kick
    ur += h * Er;
    uz += h * Ez;
    float gi = rsqrtf(1.f + (ur * ur + up * up + uz * uz) * a.inv_c2);
    const float tp = h * CB.z * gi, tz = h * a.bz * gi;
    const float sf = __fdividef(2.f, 1.f + tp * tp + tz * tz);
    const float pr = ur + (up * tz - uz * tp);   // u' = u- + u- x t, t = (0, tp, tz)
    const float pp = up - ur * tz;
    const float pz = uz + ur * tp;
    ur += sf * (pp * tz - pz * tp) + h * Er;      // u+ = u- + u' x (sf t), then half kick
    up -= sf * pr * tz;
    uz += sf * pr * tp + h * Ez;

    // move (Eq. DNE) in the ring's Cartesian frame, rotate back to the meridian plane
    gi = rsqrtf(1.f + (ur * ur + up * up + uz * uz) * a.inv_c2);
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

    // first segment, in the start triangle (the whole path for most particles)
    const float dl0 = G.x * d0 + G.y * d1, dl1 = G.z * d0 + G.w * d1;
    const Seg sg = segment_end(f0, f1, f2, dl0, dl1, -(dl0 + dl1), -1);
    currents(s0, s1, s2, sg, flags, j0a, j0b, j0c);
    if (sg.kx < 0) {
        __stcs(a.p.l0 + i, sg.e0);
        __stcs(a.p.l1 + i, sg.e1);
    } else {
        crossed = true;
        e = QEntry{i, t0, sg.kx, sg.e0, sg.e1, d0 * (1.f - sg.sx), d1 * (1.f - sg.sx)};
    }
}

// Finish a particle that reached an edge: stop on the axis, leave at a wall or at the walk
// cap (its charge goes to Q_abs), or enter the neighbour (the shared nodes keep their
// coordinates) and deposit that segment's current, repeating across further edges.
// Returns the number of crossings after the first.
__device__ __forceinline__ unsigned walk_on(const PushArgs<PF32> &a, const QEntry &q) {
    int t = q.t, kx = q.kx;
    int s0 = q.s0, s1 = q.s1, s2 = LAM_ONE - q.s0 - q.s1;
    float d0 = q.d0, d1 = q.d1;
    int4 nd = __ldg(rec4i(a.rec, t) + 4);
    int4 NB = __ldg(rec4i(a.rec, t) + 6);
    unsigned cx = 0;
    for (int ncross = 0;; ncross++) {
        const int nb = sel3(kx, NB.x, NB.y, NB.z);
        if (nb < 0 && -nb == PIC_BC_AXIS) {
            // the meridian segment stays at rho >= 0: it stops on the axis edge
            __stcs(a.p.tri + q.slot, t);
            __stcs(a.p.l0 + q.slot, s0);
            __stcs(a.p.l1 + q.slot, s1);
            return cx;
        }
        if (nb < 0 || ncross + 1 >= a.walk_cap) {
            red_add(a.Qabs + nd.x, s0);
            red_add(a.Qabs + nd.y, s1);
            red_add(a.Qabs + nd.z, s2);
            if (nb >= 0) atomicAdd(a.counters + CNT_OVERFLOW, 1ULL);
            atomicAdd(a.counters + CNT_ABSORBED, 1ULL);
            __stcs(a.p.tri + q.slot, -1);
            return cx;
        }
        const int ga = sel3(kx, nd.y, nd.z, nd.x), gb = sel3(kx, nd.z, nd.x, nd.y);
        const int va = sel3(kx, s1, s2, s0), vb = sel3(kx, s2, s0, s1);
        const float4 GN = __ldg(rec4(a.rec, nb));
        const int4 NN = __ldg(rec4i(a.rec, nb) + 4);
        const int4 EG = __ldg(rec4i(a.rec, nb) + 5);
        NB = __ldg(rec4i(a.rec, nb) + 6);
        s0 = NN.x == ga ? va : (NN.x == gb ? vb : 0);
        s1 = NN.y == ga ? va : (NN.y == gb ? vb : 0);
        s2 = NN.z == ga ? va : (NN.z == gb ? vb : 0);
        const int entered = (NN.x != ga && NN.x != gb) ? 0 : ((NN.y != ga && NN.y != gb) ? 1 : 2);
        t = nb;
        nd = NN;
        const float dl0 = GN.x * d0 + GN.y * d1, dl1 = GN.z * d0 + GN.w * d1;
        const Seg sg = segment_end(fix2f(s0), fix2f(s1), fix2f(s2), dl0, dl1, -(dl0 + dl1), entered);
        long long J0, J1, J2;
        currents(s0, s1, s2, sg, NN.w, J0, J1, J2);
        red_add(a.J + EG.x, J0);
        red_add(a.J + EG.y, J1);
        red_add(a.J + EG.z, J2);
        s0 = sg.e0;
        s1 = sg.e1;
        s2 = sg.e2;
        if (sg.kx < 0) {
            __stcs(a.p.tri + q.slot, t);
            __stcs(a.p.l0 + q.slot, s0);
            __stcs(a.p.l1 + q.slot, s1);
            return cx;
        }
        cx++;
        kx = sg.kx;
        d0 *= 1.f - sg.sx;
        d1 *= 1.f - sg.sx;
    }
}

}  // namespace

__global__ void __launch_bounds__(NT, 4) k_push_f32(PushArgs<PF32> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PushSmem &sm = *reinterpret_cast<PushSmem *>(smem_raw);
    const long long n = *a.n_slots;
    const long long ntiles = (n + TILE - 1) / TILE;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned full = 0xffffffffu;
    if ((long long)blockIdx.x >= ntiles) return;
    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            mbar_init(&sm.tile_full[s], 1);
            mbar_init(&sm.q_full[s], CW);
            mbar_init(&sm.q_empty[s], 1);
            sm.qn[s] = 0;
        }
        mbar_fence_init();
    }
    __syncthreads();
    unsigned cx = 0;

    if (warp == CW) {
        // ---- walker warp: drain the queue of tile k while the compute warps do tile k+1
        int it = 0;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
            const int qb = it & 1;
            const bool ok = mbar_wait(&sm.q_full[qb], (unsigned)(it >> 1) & 1u);
            if (__any_sync(full, !ok)) {   // leave together
                if (lane == 0) atomicAdd(a.counters + CNT_TIMEOUT, 1ULL);
                break;
            }
            const int nq = sm.qn[qb];
            for (int k = lane; k < nq; k += 32) cx += walk_on(a, sm.q[qb][k]);
            __syncwarp();
            if (lane == 0) {
                sm.qn[qb] = 0;
                mbar_arrive(&sm.q_empty[qb]);
            }
        }
    } else {
        // ---- compute warps
        if (tid == 0) issue_tile(a, sm, 0, blockIdx.x, n);
        unsigned parity = 0;   // bit s: parity of the next completion of tile_full[s]
        int stage = 0, it = 0;
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
            const long long next = tile + gridDim.x;
            if (next < ntiles && tid == 0) issue_tile(a, sm, stage ^ 1, next, n);
            const int qb = it & 1;
            bool ok = it < 2 || mbar_wait(&sm.q_empty[qb], (unsigned)((it >> 1) - 1) & 1u);
            ok = ok && mbar_wait(&sm.tile_full[stage], (parity >> stage) & 1u);
            if (compute_sync_or(!ok)) {
                if (tid == 0) {
                    // let this CTA's bulk copies land before it leaves (bounded)
                    atomicAdd(a.counters + CNT_TIMEOUT, 1ULL);
                    mbar_wait(&sm.tile_full[stage], (parity >> stage) & 1u);
                    if (next < ntiles) mbar_wait(&sm.tile_full[stage ^ 1], (parity >> (stage ^ 1)) & 1u);
                }
                break;
            }
            parity ^= 1u << stage;
            const TileBuf &b = sm.buf[stage];
            const long long base = tile * TILE;
            for (int r = 0; r < ROUNDS; r++) {
                const int k = r * PT + tid;
                const long long i = base + k;
                const int t0 = i < n ? b.tri[k] : -1;
                long long j0a = 0, j0b = 0, j0c = 0;
                bool crossed = false;
                QEntry e;
                if (t0 >= 0)
                    push_first(a, (int)i, t0, b.l0[k], b.l1[k], b.ur[k], b.up[k], b.uz[k], j0a, j0b,
                               j0c, crossed, e);
                // first-segment currents: one set of atomics per start triangle per warp
                const unsigned grp = __match_any_sync(full, t0);
                if (t0 >= 0) {
                    const int cnt = __popc(grp);
                    const long long sa = group_sum(grp, cnt, j0a);
                    const long long sb = group_sum(grp, cnt, j0b);
                    const long long sc = group_sum(grp, cnt, j0c);
                    if (lane == __ffs(grp) - 1) {
                        const int4 EG = __ldg(rec4i(a.rec, t0) + 5);
                        red_add(a.J + EG.x, sa);
                        red_add(a.J + EG.y, sb);
                        red_add(a.J + EG.z, sc);
                    }
                }
                // particles that reached an edge go to the walker's queue
                const unsigned qmask = __ballot_sync(full, crossed);
                cx += crossed ? 1u : 0u;
                int qbase = 0;
                if (lane == 0 && qmask) qbase = atomicAdd(&sm.qn[qb], __popc(qmask));
                qbase = __shfl_sync(full, qbase, 0);
                if (crossed) sm.q[qb][qbase + __popc(qmask & ((1u << lane) - 1))] = e;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.q_full[qb]);
            // every compute warp is done with buffer `stage` before thread 0 refills it
            compute_sync_or(false);
            stage ^= 1;
        }
    }
    const unsigned sx = __reduce_add_sync(full, cx);
    if (lane == 0 && sx) atomicAdd(a.counters + CNT_CROSSINGS, (unsigned long long)sx);
}

struct LaunchShape {
    int bps = 0, sms = 0;
};
static LaunchShape g_push_shape[64];

void launch_push_f32(const PushArgs<PF32> &a, int64_t n_bound, cudaStream_t s) {
    if (n_bound <= 0) return;
    const int smem = (int)sizeof(PushSmem);
    int dev = 0;
    cudaGetDevice(&dev);
    LaunchShape &ps = g_push_shape[dev & 63];
    if (ps.bps == 0) {
        cudaFuncSetAttribute(k_push_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int bps = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_push_f32, NT, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ps.bps = bps > 0 ? bps : 1;
        ps.sms = sms > 0 ? sms : 1;
    }
    const int64_t tiles = (n_bound + TILE - 1) / TILE;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)ps.sms * ps.bps);
    k_push_f32<<<(unsigned)grid, NT, smem, s>>>(a);
}

}  // namespace pic
