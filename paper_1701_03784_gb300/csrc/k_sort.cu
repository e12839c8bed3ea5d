// K2: keep particles sorted by triangle and drop removed ones (counting sort: count,
// exclusive scan, scatter).  The particle kernel's coalescing and its per-triangle
// aggregation of the scatter both rely on this order; the order of particles inside a
// triangle carries no meaning (the FP32 scatter sums are order-independent).
#include <algorithm>

#include "pic_internal.h"

namespace pic {

namespace {
constexpr int SCAN_CHUNK = 2048;  // elements per scan block (256 threads x 8)
constexpr int SORT_PER = 8;       // particles per thread in the count and scatter kernels
constexpr int SORT_CHUNK = 256 * SORT_PER;
constexpr int HT_BITS = 10;       // per-block table of the chunk's triangles
constexpr int HT = 1 << HT_BITS;
constexpr int HT_PROBES = 32;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// A block's particles are a contiguous chunk of slots, which (sorted at the previous
// re-sort, moved by a few triangles since) hold few distinct triangles: they are counted
// in shared memory (open addressing on the triangle index) and reach the global counters
// and cursors once per triangle and block.  A triangle that finds no entry within
// HT_PROBES uses the global counter directly; the count and the scatter make the same
// choice, so the totals agree either way.
struct SortTable {
    int key[HT];   // triangle, -1 free
    int cnt[HT];   // particles of the chunk in it, then the running offset
    int base[HT];  // start of the chunk's range in the sorted order
};

__device__ __forceinline__ unsigned ht_hash(int t) {
    return ((unsigned)t * 2654435761u) >> (32 - HT_BITS);
}
// entry of triangle t, inserted if absent; -1 when all probed entries hold other triangles
__device__ __forceinline__ int ht_insert(SortTable &h, int t) {
    unsigned e = ht_hash(t);
    for (int q = 0; q < HT_PROBES; q++, e = (e + 1) & (HT - 1)) {
        const int k = atomicCAS(&h.key[e], -1, t);
        if (k == -1 || k == t) return (int)e;
    }
    return -1;
}
// entry of triangle t after all insertions, or -1
__device__ __forceinline__ int ht_find(const SortTable &h, int t) {
    unsigned e = ht_hash(t);
    for (int q = 0; q < HT_PROBES; q++, e = (e + 1) & (HT - 1)) {
        const int k = h.key[e];
        if (k == t) return (int)e;
        if (k == -1) return -1;
    }
    return -1;
}

__device__ __forceinline__ void ht_clear(SortTable &h) {
    for (int e = threadIdx.x; e < HT; e += blockDim.x) {
        h.key[e] = -1;
        h.cnt[e] = 0;
    }
}
}  // namespace

template <class P>
__global__ void __launch_bounds__(256) k_count(Particles<P> p, const int64_t *n_slots,
                                               int64_t *n_old, int32_t *cnt) {
    __shared__ SortTable h;
    const int64_t n = *n_slots;
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_old = n;
    int tk[SORT_PER];   // all loads issued before any is used
#pragma unroll
    for (int k = 0; k < SORT_PER; k++) {
        const int64_t i = base + k * 256 + threadIdx.x;
        tk[k] = i < n ? __ldcs(p.tri + i) : -1;
    }
    ht_clear(h);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SORT_PER; k++) {
        const int t = tk[k];
        const unsigned grp = __match_any_sync(0xffffffffu, t);
        if (t >= 0 && lane == __ffs(grp) - 1) {
            const int e = ht_insert(h, t);
            if (e >= 0) atomicAdd(&h.cnt[e], __popc(grp));
            else atomicAdd(cnt + t, __popc(grp));
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < HT; e += 256)
        if (h.key[e] >= 0) atomicAdd(cnt + h.key[e], h.cnt[e]);
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
    __shared__ SortTable h;
    const int64_t n = *n_old;
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    // the chunk's state, loaded up front: independent loads in flight together
    int t[SORT_PER], pid[SORT_PER];
    typename P::Lam l0[SORT_PER], l1[SORT_PER];
    typename P::R ur[SORT_PER], up[SORT_PER], uz[SORT_PER];
#pragma unroll
    for (int k = 0; k < SORT_PER; k++) {
        const int64_t i = base + k * 256 + threadIdx.x;
        t[k] = i < n ? __ldcs(src.tri + i) : -1;
        if (t[k] >= 0) {
            l0[k] = __ldcs(src.l0 + i);
            l1[k] = __ldcs(src.l1 + i);
            ur[k] = __ldcs(src.ur + i);
            up[k] = __ldcs(src.up + i);
            uz[k] = __ldcs(src.uz + i);
            pid[k] = __ldcs(src.pid + i);
        }
    }
    ht_clear(h);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SORT_PER; k++) {
        const unsigned grp = __match_any_sync(full, t[k]);
        if (t[k] >= 0 && lane == __ffs(grp) - 1) {
            const int e = ht_insert(h, t[k]);
            if (e >= 0) atomicAdd(&h.cnt[e], __popc(grp));
        }
    }
    __syncthreads();
    // one range of the sorted order per triangle of the chunk
    for (int e = threadIdx.x; e < HT; e += 256) {
        const int key = h.key[e];
        if (key >= 0) h.base[e] = atomicAdd(cursor + key, h.cnt[e]);
        h.cnt[e] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SORT_PER; k++) {
        const unsigned grp = __match_any_sync(full, t[k]);
        const int leader = __ffs(grp) - 1;
        int pos = 0;
        if (t[k] >= 0 && lane == leader) {
            const int e = ht_find(h, t[k]);
            pos = e >= 0 ? h.base[e] + atomicAdd(&h.cnt[e], __popc(grp))
                         : atomicAdd(cursor + t[k], __popc(grp));
        }
        pos = __shfl_sync(full, pos, leader);
        if (t[k] < 0) continue;
        const int64_t j = (int64_t)pos + __popc(grp & lanemask_lt());
        dst.tri[j] = t[k];
        dst.l0[j] = l0[k];
        dst.l1[j] = l1[k];
        dst.ur[j] = ur[k];
        dst.up[j] = up[k];
        dst.uz[j] = uz[k];
        dst.pid[j] = pid[k];
    }
}

template <class P>
void launch_resort(Particles<P> src, Particles<P> dst, int64_t *n_slots, int64_t n_bound,
                   int64_t N2, const SortScratch &sc, cudaStream_t s) {
    cudaMemsetAsync(sc.cnt, 0, sizeof(int32_t) * (N2 + 1), s);
    int64_t *n_old = sc.n_old;
    unsigned pb = (unsigned)std::max<int64_t>(1, (n_bound + SORT_CHUNK - 1) / SORT_CHUNK);
    k_count<P><<<pb, 256, 0, s>>>(src, n_slots, n_old, sc.cnt);
    PIC_LAUNCHED();
    int64_t nblk = (N2 + SCAN_CHUNK - 1) / SCAN_CHUNK;
    k_scan_sums<<<(unsigned)nblk, 256, 0, s>>>(sc.cnt, N2, sc.blk);
    PIC_LAUNCHED();
    k_scan_top<<<1, 256, 0, s>>>(sc.blk, nblk, n_slots);
    PIC_LAUNCHED();
    k_scan_apply<<<(unsigned)nblk, 256, 0, s>>>(sc.cnt, N2, sc.blk);
    PIC_LAUNCHED();
    k_scatter<P><<<pb, 256, 0, s>>>(src, dst, n_old, sc.cnt);
    PIC_LAUNCHED();
}

template void launch_resort<PF32>(Particles<PF32>, Particles<PF32>, int64_t *, int64_t, int64_t,
                                  const SortScratch &, cudaStream_t);
template void launch_resort<PF64>(Particles<PF64>, Particles<PF64>, int64_t *, int64_t, int64_t,
                                  const SortScratch &, cudaStream_t);

}  // namespace pic
