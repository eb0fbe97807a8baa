// Binning and depth sort (the step between "preprocess" and "rasterize" in RGBAvatar Sec. 3.2;
// the paper's renderer inherits it from 3DGS): every kept Gaussian is listed in every screen
// tile of its rectangle and each (frame, tile) list is ordered by (depth bits, Gaussian index).
//
// Design: the per-tile counts come out of the preprocess kernel (atomics whose return values
// give each Gaussian its slot in up to 8 tiles), one CTA scans them into list offsets and a
// work list, a scatter kernel drops (depth << 32 | index) keys into their tile's segment (by
// slot, or by a cursor atomic for larger rectangles), and one CTA per non-empty tile sorts its
// shared memory, or through L2 for long segments (a stable LSD radix sort on the key compressed
// to (depth - segment minimum, index); a bitonic network when that key would need more than 64
// bits). Because the key carries the index, the result is unique.
#include "rgba_internal.cuh"

namespace rgba {
namespace {

constexpr int kScanThreads = 1024;

// Per tile (one thread each, coalesced): the total count into tile_start (the scan below turns
// it into the list start) and, for the larger rectangles, each sub-counter's fill offset
// relative to the tile's start (after the ranked slots).
__global__ void k_tile_totals(Ctx c) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= c.T) return;
    const unsigned *sub = c.tile_count + c.T + t * kSubCounters;
    unsigned v = c.tile_count[t];
#pragma unroll
    for (int q = 0; q < kSubCounters; ++q) {
        c.cursor[t * kSubCounters + q] = v;
        v += sub[q];
    }
    c.tile_start[t] = v;
}

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
        unsigned v = c.tile_start[t];  // the tile's total (k_tile_totals)
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
        const unsigned v = c.tile_start[t];
        unsigned st = run > 0xffffffffull ? 0xffffffffu : (unsigned)run;
        c.tile_start[t] = st;
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
    const int w = rc.z - rc.x, area = w * (rc.w - rc.y);
    if (area <= kRankSlots) {  // slots recorded by the preprocess: no atomics
        const uint4 *rp = reinterpret_cast<const uint4 *>(c.ranks + r * kRankSlots);
        const uint4 r0 = rp[0], r1 = rp[1];
        const unsigned rk[kRankSlots] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
        for (int q = 0; q < kRankSlots; ++q) {
            if (q < area) {
                const int dy = q / w;
                const long long gt = f.tile_base + (long long)(rc.y + dy) * f.tiles_x + rc.x + (q - dy * w);
                c.keys[c.tile_start[gt] + rk[q]] = key;
            }
        }
        return;
    }
    unsigned *cur = c.cursor + (r & (kSubCounters - 1));
    for (int ty = rc.y; ty < rc.w; ++ty)
        for (int tx = rc.x; tx < rc.z; ++tx) {
            const long long gt = f.tile_base + (long long)ty * f.tiles_x + tx;
            const unsigned pos = c.tile_start[gt] + atomicAdd(cur + gt * kSubCounters, 1u);
            c.keys[pos] = key;
        }
}

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadixCap = 8192;       // keys a segment may have for the shared-memory radix sort
constexpr int kSortSmemKeys = 16384;  // bitonic fallback in shared memory up to this length

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

// Stable LSD radix sort of L keys in shared memory, 8-bit digits, `bits` significant bits.
// Warp w owns the contiguous run [w S, (w+1) S) of the input; within a warp, rounds of 32 keys
// go in order and lanes are ranked by lane index among equal digits (__match_any_sync), so the
// order of equal digits is kept and the result after the last pass is fully sorted.
// Returns the buffer holding the result (a or b).
__device__ unsigned long long *radix_sort(unsigned long long *a, unsigned long long *b, int L,
                                          int bits, unsigned *s_cnt /* [warps][256] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = ((L + kSortWarps - 1) / kSortWarps + 31) & ~31;
    const int lo = warp * S, hi = min(L, lo + S);
    unsigned *cnt = s_cnt + warp * 256;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int shift = 0; shift < bits; shift += 8) {
        for (int d = lane; d < 256; d += 32) cnt[d] = 0;
        __syncwarp();
        for (int base = lo; base < hi; base += 32) {
            const int e = base + lane;
            const bool ok = e < hi;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const unsigned d = (unsigned)(a[e] >> shift) & 255u;
                const unsigned peers = __match_any_sync(act, d);
                if ((peers & lt_mask) == 0) cnt[d] += __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        // bases in (digit, warp) order: digit totals scanned, then warps in order within a digit
        if (threadIdx.x < 256) {
            const int d = threadIdx.x;
            unsigned run = 0;
            for (int w = 0; w < kSortWarps; ++w) {
                const unsigned c = s_cnt[w * 256 + d];
                s_cnt[w * 256 + d] = run;
                run += c;
            }
            s_cnt[kSortWarps * 256 + d] = run;  // digit total
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // exclusive scan of the 256 digit totals by one warp
            unsigned *tot = s_cnt + kSortWarps * 256;
            unsigned carry = 0;
            for (int c0 = 0; c0 < 256; c0 += 32) {
                const unsigned v = tot[c0 + lane];
                unsigned x = v;
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                tot[c0 + lane] = carry + x - v;
                carry += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        __syncthreads();
        for (int d = lane; d < 256; d += 32) cnt[d] += s_cnt[kSortWarps * 256 + d];
        __syncwarp();
        for (int base = lo; base < hi; base += 32) {
            const int e = base + lane;
            const bool ok = e < hi;
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            unsigned d = 0, peers = 0, pos = 0;
            unsigned long long k = 0;
            if (ok) {
                k = a[e];
                d = (unsigned)(k >> shift) & 255u;
                peers = __match_any_sync(act, d);
                pos = cnt[d] + __popc(peers & lt_mask);
            }
            __syncwarp();
            if (ok) {
                b[pos] = k;
                if ((peers & lt_mask) == 0) cnt[d] += __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        unsigned long long *t = a;
        a = b;
        b = t;
    }
    return a;
}

__global__ void __launch_bounds__(kSortThreads) k_tile_sort(Ctx c) {
    extern __shared__ unsigned long long s_keys[];  // [kRadixCap] x 2 or [kSortSmemKeys]
    unsigned *s_cnt = reinterpret_cast<unsigned *>(s_keys + 2 * kRadixCap);  // [warps + 1][256]
    __shared__ unsigned s_w, s_dmin, s_dmax, s_imax;
    if (c.cnt->overflow) return;
    const unsigned n_work = c.cnt->n_work;
    while (true) {
        if (threadIdx.x == 0) {
            s_w = atomicAdd(&c.cnt->next_sort, 1u);
            s_dmin = 0xffffffffu;
            s_dmax = 0u;
            s_imax = 0u;
        }
        __syncthreads();
        const unsigned w = s_w;
        if (w >= n_work) break;
        const unsigned t = c.work[w];
        const unsigned st = c.tile_start[t], L = c.tile_start[t + 1] - st;
        unsigned long long *g = c.keys + st;
        bool sorted = false;
        {
            // compress the key to (depth - min depth) << index bits | index
            unsigned dmin = 0xffffffffu, dmax = 0u, imax = 0u;
            for (unsigned e = threadIdx.x; e < L; e += blockDim.x) {
                const unsigned long long k = g[e];
                const unsigned d = (unsigned)(k >> 32), i = (unsigned)k;
                dmin = min(dmin, d);
                dmax = max(dmax, d);
                imax = max(imax, i);
            }
            for (int o = 16; o > 0; o >>= 1) {
                dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
                dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
                imax = max(imax, __shfl_xor_sync(0xffffffffu, imax, o));
            }
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&s_dmin, dmin);
                atomicMax(&s_dmax, dmax);
                atomicMax(&s_imax, imax);
            }
            __syncthreads();
            const unsigned d0 = s_dmin;
            const int ib = 32 - __clz(s_imax);            // bits of the largest index (0 if 0)
            const int db = 32 - __clz(s_dmax - d0);       // bits of the depth spread
            if (db + ib <= 64) {
                // in shared memory when the segment fits, else in place in global memory (L2)
                const bool in_smem = L <= (unsigned)kRadixCap;
                unsigned long long *a = in_smem ? s_keys : c.keys2 + st;
                unsigned long long *bb = in_smem ? s_keys + kRadixCap : g;
                for (unsigned e = threadIdx.x; e < L; e += blockDim.x) {
                    const unsigned long long k = g[e];
                    a[e] = ((unsigned long long)((unsigned)(k >> 32) - d0) << ib) | (unsigned)k;
                }
                __syncthreads();
                const unsigned long long *res = radix_sort(a, bb, (int)L, db + ib, s_cnt);
                const unsigned long long imask = (1ull << ib) - 1ull;
                for (unsigned e = threadIdx.x; e < L; e += blockDim.x)
                    c.sorted[st + e] = (unsigned)(res[e] & imask);
                sorted = true;
            }
        }
        if (sorted) {
        } else if (L <= (unsigned)kSortSmemKeys) {
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
    k_tile_totals<<<(unsigned)((c.T + 255) / 256), 256, 0, s>>>(c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
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
    const int smem = 2 * kRadixCap * (int)sizeof(unsigned long long) + (kSortWarps + 1) * 256 * 4;
    static_assert(2 * kRadixCap >= kSortSmemKeys, "bitonic fallback fits the radix buffers");
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
