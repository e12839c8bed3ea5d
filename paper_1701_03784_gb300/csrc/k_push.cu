// K1: fused particle step -- Whitney gather, relativistic Boris push, rotate-back to the
// meridian plane, triangle walk with segment splitting, charge-conserving scatter.
//
// One thread per particle slot, particles stored structure-of-arrays and kept sorted by
// triangle, so a warp's loads are coalesced and its triangle records are broadcast from
// L1.  Scatter (Eq. current, Eq. charge): the contributions of each particle's first
// segment and of its final charge, when it ends where it started, are summed over the
// lanes that share a triangle (match.any + redux.sync on 23-bit limbs of the int64 fixed
// point values) and one lane per triangle issues the atomics.  Segments in other triangles
// (edge crossings) go straight to global atomics.
#include <type_traits>

#include "pic_internal.h"

namespace pic {

namespace {

template <class R>
struct Vec3 {
    R r, p, z;  // (rho, phi, z) components
};

template <class R>
__device__ __forceinline__ Vec3<R> cross(const Vec3<R> &a, const Vec3<R> &b) {
    return {a.p * b.z - a.z * b.p, a.z * b.r - a.r * b.z, a.r * b.p - a.p * b.r};
}

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

// Eq. DLE with its magnetic term read as the mean of the velocities v^{n-1/2} and
// v^{n+1/2} (Vay 2008, the correction cited in Sec. 3.3), solved in closed form.  Fields in
// the local frame: E = (Er, 0, Ez), B = (0, bphi, bz); h = q dt / (2 m).
//   u' = u + 2h E + h (u / gamma(u)) x B,  tau = h B,
//   gamma_new^2 = (sigma + sqrt(sigma^2 + 4 (tau^2 + (u'.tau)^2 / c^2))) / 2,
//   sigma = gamma(u')^2 - tau^2 (the other form of the root when sigma < 0),
//   t = tau / gamma_new,  u_new = (u' + (u'.t) t + u' x t) / (1 + t^2).
template <class R>
__device__ __forceinline__ Vec3<R> kick_vay(const Vec3<R> &u, R Er, R Ez, R bphi, R bz, R h,
                                            R inv_c2) {
    const R gi = rsqrt_(R(1) + (u.r * u.r + u.p * u.p + u.z * u.z) * inv_c2);
    const R tp = h * bphi, tz = h * bz;
    const R hg = gi;
    // (u / gamma) x tau with tau = (0, tp, tz)
    const Vec3<R> p = {u.r + R(2) * h * Er + hg * (u.p * tz - u.z * tp), u.p - hg * u.r * tz,
                       u.z + R(2) * h * Ez + hg * u.r * tp};
    const R tau2 = tp * tp + tz * tz;
    const R ut0 = p.p * tp + p.z * tz;
    const R x = tau2 + ut0 * ut0 * inv_c2;
    const R sigma = R(1) + (p.r * p.r + p.p * p.p + p.z * p.z) * inv_c2 - tau2;
    const R disc = sqrt_(sigma * sigma + R(4) * x);
    const R g2 = sigma >= R(0) ? R(0.5) * (sigma + disc) : R(2) * x / (disc - sigma);
    const R gn = rsqrt_(g2);
    const R qp = tp * gn, qz = tz * gn;
    const R ut = p.p * qp + p.z * qz;
    const R sf = R(1) / (R(1) + qp * qp + qz * qz);
    return Vec3<R>{sf * (p.r + p.p * qz - p.z * qp), sf * (p.p + ut * qp - p.r * qz),
                   sf * (p.z + ut * qz + p.r * qp)};
}

// barycentric state: FP32 keeps exact integers (units 2^-22, sum 2^22) plus their float
// values; FP64 keeps doubles
template <class P>
struct Bary;

template <>
struct Bary<PF32> {
    int32_t q[3];
    float f[3];
    __device__ void set_int(int32_t a, int32_t b) {
        q[0] = a;
        q[1] = b;
        q[2] = LAM_ONE - a - b;
        for (int k = 0; k < 3; k++) f[k] = (float)q[k] * (float)LAM_INV;
    }
};
template <>
struct Bary<PF64> {
    double f[3];
};

// Round three non-negative coordinates that sum to ~1 to integers that sum to 2^22.
__device__ __forceinline__ void quantize(const float in[3], Bary<PF32> &out) {
    float a = fmaxf(in[0], 0.f), b = fmaxf(in[1], 0.f), c = fmaxf(in[2], 0.f);
    float s = a + b + c;
    float inv = (float)LAM_ONE / s;
    int32_t qa = __float2int_rn(a * inv), qb = __float2int_rn(b * inv);
    int32_t qc = LAM_ONE - qa - qb;
    if (qc < 0) {
        if (qa >= qb) qa += qc; else qb += qc;
        qc = 0;
    }
    out.q[0] = qa;
    out.q[1] = qb;
    out.q[2] = qc;
    for (int k = 0; k < 3; k++) out.f[k] = (float)out.q[k] * (float)LAM_INV;
}

// A point on local edge kx: coordinate kx is exactly 0 and the other two are integers
// that sum to 2^22 (the neighbour inherits them unchanged).
__device__ __forceinline__ void quantize_on_edge(int kx, float ci, float cj, Bary<PF32> &out) {
    const int ii = (kx + 1) % 3, jj = (kx + 2) % 3;
    ci = fmaxf(ci, 0.f);
    cj = fmaxf(cj, 0.f);
    int32_t qi = __float2int_rn(ci / (ci + cj) * (float)LAM_ONE);
    qi = min(max(qi, 0), LAM_ONE);
    out.q[kx] = 0;
    out.q[ii] = qi;
    out.q[jj] = LAM_ONE - qi;
    for (int k = 0; k < 3; k++) out.f[k] = (float)out.q[k] * (float)LAM_INV;
}

// segment current on the three edges of triangle `rec`: lam_a^s lam_b^e - lam_b^s lam_a^e
// for each local edge with tail a and head b (Eq. current as the line integral of W1)
__device__ __forceinline__ void segment_current(const int32_t flags, const Bary<PF32> &s,
                                                const Bary<PF32> &e, long long out[3]) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        int a = (flags >> k) & 1 ? i : j;
        int b = (flags >> k) & 1 ? j : i;
        out[k] = (long long)s.q[a] * e.q[b] - (long long)s.q[b] * e.q[a];
    }
}
__device__ __forceinline__ void segment_current(const int32_t flags, const Bary<PF64> &s,
                                                const Bary<PF64> &e, double out[3]) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        int a = (flags >> k) & 1 ? i : j;
        int b = (flags >> k) & 1 ? j : i;
        out[k] = s.f[a] * e.f[b] - s.f[b] * e.f[a];
    }
}

__device__ __forceinline__ void atomic_acc(unsigned long long *p, long long v) {
    if (v != 0) atomicAdd(p, (unsigned long long)v);
}
__device__ __forceinline__ void atomic_acc(double *p, double v) {
    if (v != 0.0) atomicAdd(p, v);
}

// Sum a signed int64 (|v| < 2^45) over the lanes of `grp` with 32-bit redux.sync on two
// 23-bit limbs of v + 2^45 (each limb sum stays below 2^28).
__device__ __forceinline__ long long group_sum(unsigned grp, int n, long long v) {
    const long long bias = 1LL << 45;
    unsigned long long b = (unsigned long long)(v + bias);
    unsigned lo = (unsigned)(b & 0x7FFFFFu);
    unsigned hi = (unsigned)(b >> 23);
    unsigned slo = __reduce_add_sync(grp, lo);
    unsigned shi = __reduce_add_sync(grp, hi);
    return ((long long)shi << 23) + (long long)slo - (long long)n * bias;
}

template <class P>
__device__ __forceinline__ void load_bary(const Particles<P> &p, int64_t i, Bary<P> &l);
template <>
__device__ __forceinline__ void load_bary<PF32>(const Particles<PF32> &p, int64_t i,
                                               Bary<PF32> &l) {
    l.set_int(p.l0[i], p.l1[i]);
}
template <>
__device__ __forceinline__ void load_bary<PF64>(const Particles<PF64> &p, int64_t i,
                                               Bary<PF64> &l) {
    l.f[0] = p.l0[i];
    l.f[1] = p.l1[i];
    l.f[2] = 1.0 - l.f[0] - l.f[1];
}

}  // namespace

template <class P>
__global__ void __launch_bounds__(256) k_push(PushArgs<P> a) {
    using R = typename P::R;
    using Acc = typename P::Acc;
    using Contrib = typename std::conditional<P::fixed, long long, double>::type;
    const int64_t n = *a.n_slots;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int t0 = i < n ? a.p.tri[i] : -1;

    // aggregated contributions of this lane in its start triangle t0
    Contrib j0[3] = {0, 0, 0}, q0[3] = {0, 0, 0};
    unsigned cnt_abs = 0, cnt_ovf = 0, cnt_x = 0;

    if (t0 >= 0) {
        const TriRec<R> *rc = a.rec + t0;
        Bary<P> l;
        load_bary<P>(a.p, i, l);
        // gather (Sec. 3.2): E(lambda) = sum_k lambda_k c_k; B_phi time-centred; guide B_z
        R Ez = l.f[0] * rc->c[0] + l.f[1] * rc->c[2] + l.f[2] * rc->c[4];
        R Er = l.f[0] * rc->c[1] + l.f[1] * rc->c[3] + l.f[2] * rc->c[5];
        R rho = l.f[0] * rc->rho[0] + l.f[1] * rc->rho[1] + l.f[2] * rc->rho[2];
        const R h = a.qmdt2;
        // relativistic push (Eq. DLE)
        Vec3<R> u;
        if (a.pusher == PIC_PUSHER_VAY) {
            u = kick_vay<R>(Vec3<R>{a.p.ur[i], a.p.up[i], a.p.uz[i]}, Er, Ez, rc->bphi, a.bz, h,
                            a.inv_c2);
        } else {
            // Boris: half kick, rotation by t = h B / gamma(u-), half kick
            Vec3<R> um = {a.p.ur[i] + h * Er, a.p.up[i], a.p.uz[i] + h * Ez};
            R g_inv = rsqrt_(R(1) + (um.r * um.r + um.p * um.p + um.z * um.z) * a.inv_c2);
            Vec3<R> tv = {R(0), h * rc->bphi * g_inv, h * a.bz * g_inv};
            R sfac = R(2) / (R(1) + tv.p * tv.p + tv.z * tv.z);
            Vec3<R> c1 = cross(um, tv);
            Vec3<R> upr = {um.r + c1.r, um.p + c1.p, um.z + c1.z};
            Vec3<R> c2 = cross(upr, Vec3<R>{R(0), sfac * tv.p, sfac * tv.z});
            u = Vec3<R>{um.r + c2.r + h * Er, um.p + c2.p, um.z + c2.z + h * Ez};
        }
        // move (Eq. DNE) in the ring's Cartesian frame, rotate back to the meridian plane
        R gn_inv = rsqrt_(R(1) + (u.r * u.r + u.p * u.p + u.z * u.z) * a.inv_c2);
        R xr = u.r * gn_inv * a.dt, yp = u.p * gn_inv * a.dt;
        R x = rho + xr;
        R rn2 = x * x + yp * yp;
        R rn = sqrt_(rn2);
        R drho = (rn + rho) > R(0) ? (R(2) * rho * xr + xr * xr + yp * yp) / (rn + rho) : R(0);
        if (rn > R(0)) {
            R cs = x / rn, sn = yp / rn;
            R ur = cs * u.r + sn * u.p;
            u.p = -sn * u.r + cs * u.p;
            u.r = ur;
        }
        a.p.ur[i] = u.r;
        a.p.up[i] = u.p;
        a.p.uz[i] = u.z;
        R d0 = u.z * gn_inv * a.dt, d1 = drho;

        // walk the straight meridian segment, splitting it at edge crossings
        int t = t0, entered = -1;
        int32_t flags = rc->flags;
        R g[6];
        g[0] = rc->g[0]; g[1] = rc->g[1]; g[2] = rc->g[2]; g[3] = rc->g[3];
        g[4] = -g[0] - g[2]; g[5] = -g[1] - g[3];
        bool alive = true, first = true;
        for (int ncross = 0;; ncross++) {
            R dl[3], le[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                dl[k] = g[2 * k] * d0 + g[2 * k + 1] * d1;
                le[k] = l.f[k] + dl[k];
            }
            int kx = -1;
            R sx = R(2);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (k == entered || !(le[k] < R(0))) continue;
                R s = l.f[k] / (l.f[k] - le[k]);
                if (s < sx) { sx = s; kx = k; }
            }
            Bary<P> e;
            if (kx < 0) {
                if constexpr (P::fixed) {
                    quantize(le, e);
                } else {
                    if (entered >= 0 && le[entered] < 0.0) {
                        le[entered] = 0.0;
                        int ii = (entered + 1) % 3, jj = (entered + 2) % 3;
                        double sum = le[ii] + le[jj];
                        le[ii] /= sum;
                        le[jj] /= sum;
                    }
                    for (int k = 0; k < 3; k++) e.f[k] = le[k];
                }
            } else {
                int ii = (kx + 1) % 3, jj = (kx + 2) % 3;
                R ci = l.f[ii] + sx * dl[ii], cj = l.f[jj] + sx * dl[jj];
                if constexpr (P::fixed) {
                    quantize_on_edge(kx, ci, cj, e);
                } else {
                    double sum = ci + cj;
                    e.f[kx] = 0.0;
                    e.f[ii] = ci / sum;
                    e.f[jj] = cj / sum;
                }
            }
            // scatter the segment's current (Eq. current)
            Contrib jc[3];
            segment_current(flags, l, e, jc);
            if (first) {
                j0[0] = jc[0]; j0[1] = jc[1]; j0[2] = jc[2];
                first = false;
            } else {
                const TriRec<R> *rt = a.rec + t;
#pragma unroll
                for (int k = 0; k < 3; k++) atomic_acc(a.J + rt->edge[k], jc[k]);
            }
            l = e;
            if (kx < 0) break;
            cnt_x++;
            const TriRec<R> *rt = a.rec + t;
            int nb = rt->nbr[kx];
            if (nb < 0 && -nb == PIC_BC_AXIS) break;  // stays on the axis edge
            if (nb < 0 || ncross + 1 >= a.walk_cap) {
                // absorbed at the wall (or walk cap): its charge leaves the grid
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if constexpr (P::fixed) atomic_acc(a.Qabs + rt->node[k], (long long)l.q[k]);
                    else atomic_acc(a.Qabs + rt->node[k], l.f[k]);
                }
                if (nb >= 0) cnt_ovf++;
                cnt_abs++;
                alive = false;
                break;
            }
            // enter the neighbour: the two shared nodes keep their coordinates
            int gi = rt->node[(kx + 1) % 3], gj = rt->node[(kx + 2) % 3];
            const TriRec<R> *rn_ = a.rec + nb;
            Bary<P> ln;
            int third = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                int nk = rn_->node[k];
                if constexpr (P::fixed) {
                    ln.q[k] = nk == gi ? l.q[(kx + 1) % 3] : (nk == gj ? l.q[(kx + 2) % 3] : 0);
                } else {
                    ln.f[k] = nk == gi ? l.f[(kx + 1) % 3] : (nk == gj ? l.f[(kx + 2) % 3] : 0.0);
                }
                if (nk != gi && nk != gj) third = k;
            }
            if constexpr (P::fixed) {
                for (int k = 0; k < 3; k++) ln.f[k] = (float)ln.q[k] * (float)LAM_INV;
            }
            l = ln;
            entered = third;
            d0 *= (R(1) - sx);
            d1 *= (R(1) - sx);
            t = nb;
            flags = rn_->flags;
            g[0] = rn_->g[0]; g[1] = rn_->g[1]; g[2] = rn_->g[2]; g[3] = rn_->g[3];
            g[4] = -g[0] - g[2]; g[5] = -g[1] - g[3];
        }
        // charge at the new position (Eq. charge)
        if (alive) {
            if (t == t0) {
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if constexpr (P::fixed) q0[k] = l.q[k]; else q0[k] = l.f[k];
                }
            } else {
                const TriRec<R> *rt = a.rec + t;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if constexpr (P::fixed) atomic_acc(a.Q + rt->node[k], (long long)l.q[k]);
                    else atomic_acc(a.Q + rt->node[k], l.f[k]);
                }
            }
            a.p.tri[i] = t;
            if constexpr (P::fixed) {
                a.p.l0[i] = l.q[0];
                a.p.l1[i] = l.q[1];
            } else {
                a.p.l0[i] = l.f[0];
                a.p.l1[i] = l.f[1];
            }
        } else {
            a.p.tri[i] = -1;
        }
    }

    // first-segment current and same-triangle charge: one atomic per triangle per warp
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if constexpr (P::fixed) {
        unsigned grp = __match_any_sync(full, t0);
        if (t0 >= 0) {
            int cnt = __popc(grp);
            long long s[6];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                s[k] = group_sum(grp, cnt, j0[k]);
                s[3 + k] = group_sum(grp, cnt, q0[k]);
            }
            if (lane == __ffs(grp) - 1) {
                const TriRec<R> *rc = a.rec + t0;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    atomic_acc(a.J + rc->edge[k], s[k]);
                    atomic_acc(a.Q + rc->node[k], s[3 + k]);
                }
            }
        }
    } else {
        if (t0 >= 0) {
            const TriRec<R> *rc = a.rec + t0;
            for (int k = 0; k < 3; k++) {
                atomic_acc(a.J + rc->edge[k], j0[k]);
                atomic_acc(a.Q + rc->node[k], q0[k]);
            }
        }
    }
    unsigned s_abs = __reduce_add_sync(full, cnt_abs);
    unsigned s_ovf = __reduce_add_sync(full, cnt_ovf);
    unsigned s_x = __reduce_add_sync(full, cnt_x);
    if (lane == 0) {
        if (s_abs) atomicAdd(a.counters + CNT_ABSORBED, (unsigned long long)s_abs);
        if (s_ovf) atomicAdd(a.counters + CNT_OVERFLOW, (unsigned long long)s_ovf);
        if (s_x) atomicAdd(a.counters + CNT_CROSSINGS, (unsigned long long)s_x);
    }
}

template <class P>
void launch_push(const PushArgs<P> &a, int64_t n_bound, cudaStream_t s) {
    if constexpr (P::fixed) {
        launch_push_f32(a, n_bound, s);
    } else {
        if (n_bound <= 0) return;
        int64_t blocks = (n_bound + 255) / 256;
        k_push<P><<<(unsigned)blocks, 256, 0, s>>>(a);
        PIC_LAUNCHED();
    }
}

// Eq. charge of the particles in slots [first, first + count) (new particles at
// injection; all of them for the diagnostics).  FP32 build: the fixed-point coordinates of
// the lanes that share a triangle are summed first (sorted slots: most lanes of a warp do),
// one set of atomics per triangle; sums of at most 32 coordinates < 2^23 fit in 32 bits.
template <class P>
__global__ void k_deposit_q(const TriRec<typename P::R> *rec, Particles<P> p, int64_t first,
                            int64_t count, typename P::Acc *Q) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = first + k;
    const int t = k < count ? p.tri[i] : -1;
    if constexpr (P::fixed) {
        const unsigned grp = __match_any_sync(0xffffffffu, t);
        if (t < 0) return;
        const unsigned a = (unsigned)p.l0[i], b = (unsigned)p.l1[i];
        const unsigned sa = __reduce_add_sync(grp, a), sb = __reduce_add_sync(grp, b);
        if ((threadIdx.x & 31) == __ffs(grp) - 1) {
            const long long sc = (long long)__popc(grp) * LAM_ONE - (long long)sa - (long long)sb;
            atomic_acc(Q + rec[t].node[0], (long long)sa);
            atomic_acc(Q + rec[t].node[1], (long long)sb);
            atomic_acc(Q + rec[t].node[2], sc);
        }
    } else {
        if (t < 0) return;
        Bary<P> l;
        load_bary<P>(p, i, l);
        for (int m = 0; m < 3; m++) atomic_acc(Q + rec[t].node[m], l.f[m]);
    }
}

template <class P>
void launch_deposit_q(const TriRec<typename P::R> *rec, Particles<P> p, int64_t first,
                      int64_t count, typename P::Acc *Q, cudaStream_t s) {
    if (count <= 0) return;
    k_deposit_q<P><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(rec, p, first, count, Q);
    PIC_LAUNCHED();
}

template void launch_push<PF32>(const PushArgs<PF32> &, int64_t, cudaStream_t);
template void launch_push<PF64>(const PushArgs<PF64> &, int64_t, cudaStream_t);
template void launch_deposit_q<PF32>(const TriRec<float> *, Particles<PF32>, int64_t, int64_t,
                                     unsigned long long *, cudaStream_t);
template void launch_deposit_q<PF64>(const TriRec<double> *, Particles<PF64>, int64_t, int64_t,
                                     double *, cudaStream_t);

}  // namespace pic
