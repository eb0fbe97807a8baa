// Binning and depth sort (the step between "preprocess" and "rasterize" in RGBAvatar Sec. 3.2;
// the paper's renderer inherits it from 3DGS): every kept Gaussian is listed in every screen
// tile of its rectangle and each (frame, tile) list is ordered by (depth bits, Gaussian index).
//
// Design: the per-tile counts come out of the preprocess kernel (atomics), one CTA scans them
// into list offsets and a work list, a scatter kernel drops (depth << 32 | index) keys into
// their tile's segment in arbitrary order, and one CTA per non-empty tile sorts its segment in
// shared memory. Because the key carries the index, the result is unique (no stability needed).
#include "rgba_internal.cuh"

namespace rgba {
namespace {

constexpr int kScanThreads = 1024;

// Exclusive scan of the tile counts (frame-major), pair total and capacity check, and the work
// list: non-empty tiles first, longest lists first (bucketed by floor(log2(length))), then the
// empty tiles in tile order. The persistent kernels pull items in this order, so the heaviest
// tiles start first and the tail of the launch is short.
__global__ void __launch_bounds__(kScanThreads) k_scan(Ctx c) {
    __shared__ unsigned long long s_sum[kScanThreads];
    __shared__ unsigned s_ne[kScanThreads];
    __shared__ unsigned s_hist[32];
    const long long T = c.T;
    const int tid = threadIdx.x;
    const long long per = (T + kScanThreads - 1) / kScanThreads;
    const long long lo = tid * per, hi = (lo + per < T) ? lo + per : T;
    if (tid < 32) s_hist[tid] = 0;
    __syncthreads();
    unsigned long long sum = 0;
    unsigned ne = 0;
    for (long long t = lo; t < hi; ++t) {
        unsigned v = c.tile_count[t];
        sum += v;
        ne += v > 0;
        if (v > 0) atomicAdd(&s_hist[31 - __clz(v)], 1u);
    }
    s_sum[tid] = sum;
    s_ne[tid] = ne;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 partials
    for (int off = 1; off < kScanThreads; off <<= 1) {
        unsigned long long a = tid >= off ? s_sum[tid - off] : 0ull;
        unsigned b = tid >= off ? s_ne[tid - off] : 0u;
        __syncthreads();
        s_sum[tid] += a;
        s_ne[tid] += b;
        __syncthreads();
    }
    if (tid == 0) {  // bucket offsets, longest bucket first
        unsigned off = 0;
        for (int k = 31; k >= 0; --k) {
            const unsigned h = s_hist[k];
            s_hist[k] = off;
            off += h;
        }
    }
    __syncthreads();
    const unsigned long long total = s_sum[kScanThreads - 1];
    const unsigned n_ne = s_ne[kScanThreads - 1];
    unsigned long long run = s_sum[tid] - sum;
    unsigned ne_run = s_ne[tid] - ne;
    unsigned e_run = (unsigned)lo - ne_run;  // empty tiles before lo
    for (long long t = lo; t < hi; ++t) {
        unsigned v = c.tile_count[t];
        unsigned st = run > 0xffffffffull ? 0xffffffffu : (unsigned)run;
        c.tile_start[t] = st;
        c.cursor[t] = st;
        if (v > 0) c.work[atomicAdd(&s_hist[31 - __clz(v)], 1u)] = (unsigned)t;
        else c.work[n_ne + e_run++] = (unsigned)t;
        run += v;
    }
    if (tid == 0) {
        c.tile_start[T] = total > 0xffffffffull ? 0xffffffffu : (unsigned)total;
        c.cnt->pairs = total > 0xffffffffull ? 0xffffffffu : (unsigned)total;
        c.cnt->overflow = total > (unsigned long long)c.cap ? 1u : 0u;
        c.cnt->n_work = n_ne;
    }
}

constexpr int kScatterThreads = 128;

__global__ void __launch_bounds__(kScatterThreads) k_scatter(Ctx c) {
    if (c.cnt->overflow) return;
    const int b = blockIdx.y;
    const FrameInfo f = c.frames[b];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    const long long r = f.rec_base + i;
    const ushort4 rc = c.rects[r];
    if (rc.z <= rc.x || rc.w <= rc.y) return;
    const unsigned bits = __float_as_uint(c.records[r * 3 + 2].y);
    const unsigned long long key = ((unsigned long long)bits << 32) | (unsigned)i;
    for (int ty = rc.y; ty < rc.w; ++ty)
        for (int tx = rc.x; tx < rc.z; ++tx) {
            const long long gt = f.tile_base + (long long)ty * f.tiles_x + tx;
            const unsigned pos = atomicAdd(c.cursor + gt, 1u);
            c.keys[pos] = key;
        }
}

constexpr int kSortThreads = 512;
constexpr int kSortSmemKeys = 16384;  // 128 KiB of keys per CTA

// Ascending bitonic network without direction flags (each merge opens with a mirrored compare),
// over a virtual power-of-two length whose entries past L are +inf: a compare whose upper
// index is >= L is skipped, so any L works and the padding never moves.
__device__ void bitonic_sort(unsigned long long *k, int L) {
    int N = 1;
    while (N < L) N <<= 1;
    for (int size = 2; size <= N; size <<= 1) {
        for (int j = size >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < (N >> 1); p += blockDim.x) {
                int blk = p / j, off = p - blk * j, i, q;
                if (j == (size >> 1)) {
                    i = blk * size + off;
                    q = blk * size + size - 1 - off;
                } else {
                    i = blk * 2 * j + off;
                    q = i + j;
                }
                if (q < L) {
                    unsigned long long a = k[i], bq = k[q];
                    if (a > bq) {
                        k[i] = bq;
                        k[q] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_tile_sort(Ctx c) {
    extern __shared__ unsigned long long s_keys[];
    __shared__ unsigned s_w;
    if (c.cnt->overflow) return;
    const unsigned n_work = c.cnt->n_work;
    while (true) {
        if (threadIdx.x == 0) s_w = atomicAdd(&c.cnt->next_sort, 1u);
        __syncthreads();
        const unsigned w = s_w;
        __syncthreads();
        if (w >= n_work) break;
        const unsigned t = c.work[w];
        const unsigned st = c.tile_start[t], L = c.tile_start[t + 1] - st;
        unsigned long long *g = c.keys + st;
        if (L <= (unsigned)kSortSmemKeys) {
            for (unsigned e = threadIdx.x; e < L; e += blockDim.x) s_keys[e] = g[e];
            __syncthreads();
            bitonic_sort(s_keys, (int)L);
            for (unsigned e = threadIdx.x; e < L; e += blockDim.x)
                c.sorted[st + e] = (unsigned)(s_keys[e] & 0xffffffffull);
        } else {
            // oversized list: the same network in place in global memory
            bitonic_sort(g, (int)L);
            for (unsigned e = threadIdx.x; e < L; e += blockDim.x)
                c.sorted[st + e] = (unsigned)(g[e] & 0xffffffffull);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_scan(const Ctx &c, cudaStream_t s) {
    k_scan<<<1, kScanThreads, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Ctx &c, int max_n, cudaStream_t s) {
    if (c.B == 0 || max_n == 0) return cudaSuccess;
    dim3 grid((max_n + kScatterThreads - 1) / kScatterThreads, c.B);
    k_scatter<<<grid, kScatterThreads, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_tile_sort(const Ctx &c, int grid, cudaStream_t s) {
    static int attr_device = -1;
    const int smem = kSortSmemKeys * (int)sizeof(unsigned long long);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_device != dev) {
        e = cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    k_tile_sort<<<grid, kSortThreads, smem, s>>>(c);
    return cudaGetLastError();
}

}  // namespace rgba
