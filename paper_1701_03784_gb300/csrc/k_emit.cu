// Cathode emission (Secs. 5.2, 5.3: electrons leave the cathode every step).  One block
// appends per_step particles behind the live slots at the start of a step, before the
// particle kernel: positions on the line z = const, uniform in area over [rho0, rho1];
// momenta u = gamma v with normal components of spread u_thermal about (0, 0, u_normal).
// Their charge (Eq. charge at the birth point) is added to Q^n, so that Eq. DCE holds for
// the step, and taken out of the Gauss-law bookkeeping (it appears without a current).
//
// Draws are counter-based: for particle id p and draw j, splitmix64(seed + 8 p + j)
// (the output function of Steele, Lea and Flood's generator, as Vigna publishes it), as a
// double in (0, 1); Box-Muller on draws 1, 2 and 3, 4.
#include <cmath>

#include "pic_internal.h"

namespace pic {

namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double unit_draw(unsigned long long seed, long long pid, int j) {
    const unsigned long long x = seed + 8ULL * (unsigned long long)pid + (unsigned long long)j;
    return ((double)(splitmix64(x) >> 11) + 0.5) * 0x1.0p-53;
}

constexpr int EMIT_THREADS = 256;

template <class P>
__global__ void __launch_bounds__(EMIT_THREADS) k_emit(EmitArgs<P> a) {
    __shared__ long long base_slot, base_pid;
    __shared__ int room;
    if (threadIdx.x == 0) {
        base_slot = *a.n_slots;
        base_pid = (long long)a.counters[CNT_NEXT_PID];
        room = base_slot + a.per_step <= a.cap;
        if (!room) atomicAdd(a.counters + CNT_EMIT_DROPPED, (unsigned long long)a.per_step);
    }
    __syncthreads();
    if (!room) return;
    const double two_pi = 6.283185307179586476925286766559;
    for (long long k = threadIdx.x; k < a.per_step; k += EMIT_THREADS) {
        const long long pid = base_pid + k;
        double u[5];
#pragma unroll
        for (int j = 0; j < 5; j++) u[j] = unit_draw(a.seed, pid, j);
        const double rho = sqrt(a.rho0 * a.rho0 + u[0] * (a.rho1 * a.rho1 - a.rho0 * a.rho0));
        // the interval of the emission line that holds rho (intervals sorted and contiguous)
        int lo = 0, hi = a.line.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.line.rho_b[mid] < rho) lo = mid + 1;
            else hi = mid;
        }
        const double ra = a.line.rho_a[lo], rb = a.line.rho_b[lo];
        const double s = fmin(fmax((rho - ra) / (rb - ra), 0.0), 1.0);
        double lam[3];
#pragma unroll
        for (int m = 0; m < 3; m++) {
            const double la = a.line.lam_a[3 * lo + m], lb = a.line.lam_b[3 * lo + m];
            lam[m] = fmax(la + s * (lb - la), 0.0);
        }
        const int t = a.line.tri[lo];
        const double r1 = sqrt(-2.0 * log(u[1])), r3 = sqrt(-2.0 * log(u[3]));
        const double ur = a.u_thermal * r1 * cos(two_pi * u[2]);
        const double up = a.u_thermal * r1 * sin(two_pi * u[2]);
        const double uz = a.u_normal + a.u_thermal * r3 * cos(two_pi * u[4]);
        const long long i = base_slot + k;
        a.p.tri[i] = t;
        a.p.ur[i] = (typename P::R)ur;
        a.p.up[i] = (typename P::R)up;
        a.p.uz[i] = (typename P::R)uz;
        a.p.pid[i] = (int32_t)pid;
        const int4 nd = make_int4(a.rec[t].node[0], a.rec[t].node[1], a.rec[t].node[2], 0);
        const int node[3] = {nd.x, nd.y, nd.z};
        if constexpr (P::fixed) {
            // integers that sum to 2^22 (the rule of host-side injection)
            const double ss = lam[0] + lam[1] + lam[2];
            int q0 = (int)rint(lam[0] / ss * LAM_ONE), q1 = (int)rint(lam[1] / ss * LAM_ONE);
            int q2 = LAM_ONE - q0 - q1;
            if (q2 < 0) {
                if (q0 >= q1) q0 += q2;
                else q1 += q2;
                q2 = 0;
            }
            a.p.l0[i] = q0;
            a.p.l1[i] = q1;
            const long long q[3] = {q0, q1, q2};
#pragma unroll
            for (int m = 0; m < 3; m++) {
                atomicAdd(a.Qn + node[m], (unsigned long long)q[m]);
                atomicAdd(a.Qwall + node[m], (unsigned long long)(-q[m]));
            }
        } else {
            const double ss = lam[0] + lam[1] + lam[2];
            const double l[3] = {lam[0] / ss, lam[1] / ss, lam[2] / ss};
            a.p.l0[i] = l[0];
            a.p.l1[i] = l[1];
#pragma unroll
            for (int m = 0; m < 3; m++) {
                atomicAdd(a.Qn + node[m], l[m]);
                atomicAdd(a.Qwall + node[m], -l[m]);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *a.n_slots = base_slot + a.per_step;
        a.counters[CNT_EMITTED] += (unsigned long long)a.per_step;
        a.counters[CNT_NEXT_PID] += (unsigned long long)a.per_step;
    }
}

}  // namespace

template <class P>
void launch_emit(const EmitArgs<P> &a, cudaStream_t s) {
    if (a.per_step <= 0 || a.line.n <= 0) return;
    k_emit<P><<<1, EMIT_THREADS, 0, s>>>(a);
    PIC_LAUNCHED();
}

template void launch_emit<PF32>(const EmitArgs<PF32> &, cudaStream_t);
template void launch_emit<PF64>(const EmitArgs<PF64> &, cudaStream_t);

}  // namespace pic
