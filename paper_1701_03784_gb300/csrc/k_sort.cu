// K2: keep particles sorted by triangle and drop removed ones (counting sort: count,
// exclusive scan, scatter).  The particle kernel's coalescing and its per-triangle
// aggregation of the scatter both rely on this order; the order of particles inside a
// triangle carries no meaning (the FP32 scatter sums are order-independent).
#include <algorithm>

#include "pic_internal.h"

namespace pic {

namespace {
constexpr int SCAN_CHUNK = 2048;  // elements per scan block (256 threads x 8)

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
}  // namespace

template <class P>
__global__ void __launch_bounds__(256) k_count(Particles<P> p, const int64_t *n_slots,
                                               int64_t *n_old, int32_t *cnt) {
    int64_t n = *n_slots;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *n_old = n;
    int t = i < n ? p.tri[i] : -1;
    unsigned grp = __match_any_sync(0xffffffffu, t);
    if (t >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(cnt + t, (int)__popc(grp));
}

// per-chunk sums
__global__ void __launch_bounds__(256) k_scan_sums(const int32_t *cnt, int64_t N, int32_t *blk) {
    __shared__ int32_t red[256];
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    int32_t s = 0;
    for (int k = threadIdx.x; k < SCAN_CHUNK; k += 256) {
        int64_t j = base + k;
        if (j < N) s += cnt[j];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) blk[blockIdx.x] = red[0];
}

// exclusive scan of the chunk sums (one block, sequential over 256-wide tiles); writes the
// total live count
__global__ void __launch_bounds__(256) k_scan_top(int32_t *blk, int64_t nblk, int64_t *n_slots) {
    __shared__ int32_t sh[256];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nblk; b0 += 256) {
        int64_t j = b0 + threadIdx.x;
        int32_t v = j < nblk ? blk[j] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = 1; w < 256; w <<= 1) {
            int32_t x = threadIdx.x >= w ? sh[threadIdx.x - w] : 0;
            __syncthreads();
            sh[threadIdx.x] += x;
            __syncthreads();
        }
        if (j < nblk) blk[j] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 255) carry += sh[255];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_slots = carry;
}

// exclusive scan inside each chunk plus the chunk's offset; the result is the write
// cursor of each triangle
__global__ void __launch_bounds__(256) k_scan_apply(int32_t *cnt, int64_t N, const int32_t *blk) {
    __shared__ int32_t sh[256];
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * 8;
    int32_t v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        v[k] = base + k < N ? cnt[base + k] : 0;
        s += v[k];
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 1; w < 256; w <<= 1) {
        int32_t x = threadIdx.x >= w ? sh[threadIdx.x - w] : 0;
        __syncthreads();
        sh[threadIdx.x] += x;
        __syncthreads();
    }
    int32_t run = blk[blockIdx.x] + sh[threadIdx.x] - s;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (base + k < N) cnt[base + k] = run;
        run += v[k];
    }
}

template <class P>
__global__ void __launch_bounds__(256) k_scatter(Particles<P> src, Particles<P> dst,
                                                 const int64_t *n_old, int32_t *cursor) {
    int64_t n = *n_old;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int t = i < n ? src.tri[i] : -1;
    unsigned grp = __match_any_sync(0xffffffffu, t);
    int leader = __ffs(grp) - 1;
    int base = 0;
    if (t >= 0 && (threadIdx.x & 31) == leader) base = atomicAdd(cursor + t, (int)__popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (t < 0) return;
    int64_t j = base + __popc(grp & lanemask_lt());
    dst.tri[j] = t;
    dst.l0[j] = src.l0[i];
    dst.l1[j] = src.l1[i];
    dst.ur[j] = src.ur[i];
    dst.up[j] = src.up[i];
    dst.uz[j] = src.uz[i];
    dst.pid[j] = src.pid[i];
}

template <class P>
void launch_resort(Particles<P> src, Particles<P> dst, int64_t *n_slots, int64_t n_bound,
                   int64_t N2, const SortScratch &sc, cudaStream_t s) {
    cudaMemsetAsync(sc.cnt, 0, sizeof(int32_t) * (N2 + 1), s);
    int64_t *n_old = sc.n_old;
    unsigned pb = (unsigned)std::max<int64_t>(1, (n_bound + 255) / 256);
    k_count<P><<<pb, 256, 0, s>>>(src, n_slots, n_old, sc.cnt);
    int64_t nblk = (N2 + SCAN_CHUNK - 1) / SCAN_CHUNK;
    k_scan_sums<<<(unsigned)nblk, 256, 0, s>>>(sc.cnt, N2, sc.blk);
    k_scan_top<<<1, 256, 0, s>>>(sc.blk, nblk, n_slots);
    k_scan_apply<<<(unsigned)nblk, 256, 0, s>>>(sc.cnt, N2, sc.blk);
    k_scatter<P><<<pb, 256, 0, s>>>(src, dst, n_old, sc.cnt);
}

template void launch_resort<PF32>(Particles<PF32>, Particles<PF32>, int64_t *, int64_t, int64_t,
                                  const SortScratch &, cudaStream_t);
template void launch_resort<PF64>(Particles<PF64>, Particles<PF64>, int64_t *, int64_t, int64_t,
                                  const SortScratch &, cudaStream_t);

}  // namespace pic
