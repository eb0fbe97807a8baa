// Binning and depth sort (the step between "preprocess" and "rasterize" in RGBAvatar Sec. 3.2;
// the paper's renderer inherits it from 3DGS): every kept Gaussian is listed in every screen
// tile of its rectangle and each (frame, tile) list is ordered by (depth bits, Gaussian index).
//
// Design: the per-tile counts come out of the preprocess kernel (atomics whose return values
// give each Gaussian its slot in up to 8 tiles), a three-phase scan (per-CTA partials, one CTA
// over the partials, per-CTA writes) turns them into list offsets and a work list, a scatter
// kernel drops (depth << 32 | index) keys into their tile's segment (by
// slot, or by a cursor atomic for larger rectangles), and one CTA per non-empty tile sorts its
// list, with the key compressed to (depth - segment minimum) << 32 | index: in shared memory by
// one bucket pass on the top depth bits and a placement of every key by its rank in its bucket,
// or, for long segments, through L2 by a stable LSD radix sort over the depth bits and a pass
// that orders runs of equal depth by index. Because the key carries the index, the result is
// unique.
#include "rgba_internal.cuh"

namespace rgba {
namespace {

constexpr int kScanTile = 1024;  // tiles per CTA of the three-phase scan

// Exclusive scan over the CTA (kScanTile threads) of one (u64 value, u32 count) pair per
// thread: warp shuffles, then the 32 warp totals scanned by warp 0. Also returns the totals.
__device__ __forceinline__ void block_scan(unsigned long long v, unsigned e, unsigned long long &ex_v,
                                           unsigned &ex_e, unsigned long long &tot_v, unsigned &tot_e) {
    __shared__ unsigned long long s_v[32];
    __shared__ unsigned s_e[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long xv = v;
    unsigned xe = e;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long yv = __shfl_up_sync(0xffffffffu, xv, o);
        const unsigned ye = __shfl_up_sync(0xffffffffu, xe, o);
        if (lane >= o) {
            xv += yv;
            xe += ye;
        }
    }
    if (lane == 31) {
        s_v[warp] = xv;
        s_e[warp] = xe;
    }
    __syncthreads();
    if (warp == 0) {
        unsigned long long wv = s_v[lane];
        unsigned we = s_e[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yv = __shfl_up_sync(0xffffffffu, wv, o);
            const unsigned ye = __shfl_up_sync(0xffffffffu, we, o);
            if (lane >= o) {
                wv += yv;
                we += ye;
            }
        }
        s_v[lane] = wv;
        s_e[lane] = we;
    }
    __syncthreads();
    ex_v = (warp ? s_v[warp - 1] : 0ull) + xv - v;
    ex_e = (warp ? s_e[warp - 1] : 0u) + xe - e;
    tot_v = s_v[31];
    tot_e = s_e[31];
    __syncthreads();  // s_v / s_e free for the next call
}

// The scan's per-CTA partials: [nb] sums, [nb] non-empty counts, [nb][32] bucket counts and
// the [32] bucket offsets, in the workspace.
struct ScanAux {
    unsigned long long *bsum;
    unsigned *bne, *bhist, *bucket;
};

__device__ __forceinline__ ScanAux scan_aux(const Ctx &c) {
    const long long nb = (c.T + kScanTile - 1) / kScanTile;
    ScanAux a;
    a.bsum = reinterpret_cast<unsigned long long *>(c.scan_aux);
    a.bne = reinterpret_cast<unsigned *>(a.bsum + nb);
    a.bhist = a.bne + nb;
    a.bucket = a.bhist + nb * 32;
    return a;
}

__device__ __forceinline__ unsigned bucket_of(unsigned v) { return 31u - __clz(v); }

// Phase 1, one thread per tile: the tile's total count (ranked slots plus sub-counters) into
// tile_start, each sub-counter's fill offset into cursor, and per CTA the sum, the number of
// non-empty tiles and the histogram of floor(log2(length)).
__global__ void __launch_bounds__(kScanTile) k_scan_blocks(Ctx c) {
    __shared__ unsigned s_hist[32];
    pdl_enter();
    const ScanAux a = scan_aux(c);
    if (threadIdx.x < 32) s_hist[threadIdx.x] = 0;
    __syncthreads();
    const long long t = (long long)blockIdx.x * kScanTile + threadIdx.x;
    unsigned v = 0;
    if (t < c.T) {
        const unsigned *sub = c.tile_count + tc_sub_base(c.tc_mask) + t * kSubCounters;
        v = c.tile_count[tc_word(c.tc_mask, t)];
#pragma unroll
        for (int q = 0; q < kSubCounters; ++q) {
            c.cursor[t * kSubCounters + q] = v;
            v += sub[q];
        }
        c.tile_start[t] = v;
        if (v) atomicAdd(&s_hist[bucket_of(v)], 1u);
    }
    unsigned long long ex, tot;
    unsigned exe, tote;
    block_scan(v, v > 0, ex, exe, tot, tote);
    if (threadIdx.x == 0) {
        a.bsum[blockIdx.x] = tot;
        a.bne[blockIdx.x] = tote;
    }
    if (threadIdx.x < 32) a.bhist[blockIdx.x * 32 + threadIdx.x] = s_hist[threadIdx.x];
}

// Phase 2, one CTA: exclusive scans over the CTAs of phase 1 (sums, non-empty counts, and per
// bucket the counts, warp w taking bucket w), the bucket offsets with the longest bucket first,
// the pair total, the capacity check and the work-list length.
__global__ void __launch_bounds__(kScanTile) k_scan_top(Ctx c) {
    __shared__ unsigned s_btot[32];
    pdl_enter();
    const ScanAux a = scan_aux(c);
    const long long nb = (c.T + kScanTile - 1) / kScanTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    unsigned carry_e = 0;
    for (long long b0 = 0; b0 < nb; b0 += kScanTile) {
        const long long b = b0 + threadIdx.x;
        const unsigned long long v = b < nb ? a.bsum[b] : 0ull;
        const unsigned e = b < nb ? a.bne[b] : 0u;
        unsigned long long ex, tot;
        unsigned exe, tote;
        block_scan(v, e, ex, exe, tot, tote);
        if (b < nb) {
            a.bsum[b] = carry + ex;
            a.bne[b] = carry_e + exe;
        }
        carry += tot;
        carry_e += tote;
    }
    {
        unsigned run = 0;  // warp w: bucket w, lane = CTA within a chunk of 32
        for (long long b0 = 0; b0 < nb; b0 += 32) {
            const long long b = b0 + lane;
            const unsigned h = b < nb ? a.bhist[b * 32 + warp] : 0u;
            unsigned x = h;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (b < nb) a.bhist[b * 32 + warp] = run + x - h;
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) s_btot[warp] = run;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned off = 0;
        for (int k = 31; k >= 0; --k) {
            a.bucket[k] = off;
            off += s_btot[k];
        }
        c.tile_start[c.T] = carry > 0xffffffffull ? 0xffffffffu : (unsigned)carry;
        c.cnt->pairs = carry > 0xffffffffull ? 0xffffffffu : (unsigned)carry;
        c.cnt->overflow = carry > (unsigned long long)c.cap ? 1u : 0u;
        c.cnt->n_work = carry_e;
    }
}

// Phase 3, one thread per tile: the list start (exclusive scan of the totals) and the tile's
// place in the work list: non-empty tiles by bucket, longest bucket first (in any order within
// a bucket), then the empty tiles in tile order.
__global__ void __launch_bounds__(kScanTile) k_scan_write(Ctx c) {
    __shared__ unsigned s_off[32];
    pdl_enter();
    const ScanAux a = scan_aux(c);
    const long long t = (long long)blockIdx.x * kScanTile + threadIdx.x;
    const unsigned v = t < c.T ? c.tile_start[t] : 0u;
    if (threadIdx.x < 32) s_off[threadIdx.x] = a.bucket[threadIdx.x] + a.bhist[blockIdx.x * 32 + threadIdx.x];
    const bool empty = t < c.T && v == 0;
    unsigned long long ex, tot;
    unsigned exe, tote;
    block_scan(v, empty, ex, exe, tot, tote);  // its syncs also publish s_off
    if (t < c.T) {
        const unsigned long long st = a.bsum[blockIdx.x] + ex;
        c.tile_start[t] = st > 0xffffffffull ? 0xffffffffu : (unsigned)st;
        if (v) {
            c.work[atomicAdd(&s_off[bucket_of(v)], 1u)] = (unsigned)t;
        } else {
            // empty tiles before this CTA: its first tile index minus the non-empty ones
            const unsigned e0 = (unsigned)((long long)blockIdx.x * kScanTile) - a.bne[blockIdx.x];
            c.work[c.cnt->n_work + e0 + exe] = (unsigned)t;
        }
    }
}

constexpr int kScatterThreads = 128;

__global__ void __launch_bounds__(kScatterThreads) k_scatter(Ctx c) {
    pdl_enter();
    if (c.cnt->overflow) return;
    const int b = blockIdx.y;
    const FrameInfo f = c.frames[b];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.n) return;
    const long long r = f.rec_base + i;
    const ushort4 rc = c.rects[r];
    if (rc.z <= rc.x || rc.w <= rc.y) return;
    const unsigned bits = __float_as_uint(c.depth[r]);
    const unsigned long long key = ((unsigned long long)bits << 32) | (unsigned)i;
    const int w = rc.z - rc.x, area = w * (rc.w - rc.y);
    if (area <= kRankSlots) {  // slots recorded by the preprocess: no atomics
        const uint4 *rp = reinterpret_cast<const uint4 *>(c.ranks + r * kRankSlots);
        const uint4 r0 = rp[0], r1 = rp[1];
        const unsigned rk[kRankSlots] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        const unsigned *ts = c.tile_start + f.tile_base + (long long)rc.y * f.tiles_x + rc.x;
        int ox = 0, off = 0;  // slot q is tile (rc.x + ox, rc.y + q / w), off its offset from ts
#pragma unroll
        for (int q = 0; q < kRankSlots; ++q) {
            if (q < area) {
                c.keys[ts[off] + rk[q]] = key;
                ++off;
                if (++ox == w) {
                    ox = 0;
                    off += f.tiles_x - w;
                }
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

// Asynchronous 8-byte copy global -> shared (both addresses 8-byte aligned), completed by
// cp.async.wait_all.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                 :: "r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))), "l"(src) : "memory");
}

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadixCap = 8192;                  // keys a segment may have for the shared-memory radix sort
constexpr int kMidCap = 3 * kRadixCap / 2;       // keys a segment may have for the position bucket sort
// the position sort's keys, ranks and positions fill the key area and rank array of the
// shared-memory sort exactly, so the kernel needs no more shared memory than that one: a larger
// footprint kept the next kernel's CTAs from starting on the SMs early and cost 0.12 ms per
// training step in the captured graph
static_assert(kMidCap * (8 + 2 + 2) <= kRadixCap * (2 * 8 + 2), "position sort fits the key area and rank array");
constexpr int kDigitParts = kSortThreads / 256;  // threads sharing one digit's column of warp counts
static_assert(kSortThreads % 256 == 0 && 32 % kDigitParts == 0, "whole digits per warp");

// Lanes of `act` holding the same 8-bit digit as this lane: one ballot per digit bit (a warp
// multi-split), all on the full-rate vote path.
__device__ __forceinline__ unsigned digit_peers(unsigned act, unsigned d) {
    unsigned m = act;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const unsigned bit = (d >> b) & 1u;
        const unsigned v = __ballot_sync(act, bit);
        m &= bit ? v : ~v;
    }
    return m;
}

// Stable LSD radix sort of L keys on the bits [shift0, shift_end), 8-bit digits; a and b are both in
// shared memory or both in global memory. Warp w owns the contiguous run [w S, (w+1) S) of the
// input; within a warp, rounds of 32 keys go in order and lanes are ranked by lane index among
// equal digits (digit_peers), so the order of equal digits is kept and the result after the
// last pass is fully sorted. With kCacheRanks each key's rank within its warp's run of equal
// digits is kept from the counting sweep (s_rank, L entries) and the scatter sweep only adds the
// digit base; without it the scatter sweep ranks again. Returns the buffer holding the result.
constexpr int kRounds = 4;  // rounds of 32 keys whose loads the radix sweeps issue together

template <bool kCacheRanks>
__device__ unsigned long long *radix_sort(unsigned long long *a, unsigned long long *b, int L,
                                          int shift0, int shift_end,
                                          unsigned *s_cnt /* [warps][256] + [warps] */,
                                          unsigned short *s_rank) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = ((L + kSortWarps - 1) / kSortWarps + 31) & ~31;
    const int lo = warp * S, hi = min(L, lo + S);
    unsigned *cnt = s_cnt + warp * 256;
    unsigned *wsum = s_cnt + kSortWarps * 256;
    const unsigned lt_mask = (1u << lane) - 1u;
    // thread (digit d, part q) owns the counts of digit d in warps [q W/P, (q+1) W/P)
    const int d_own = threadIdx.x / kDigitParts, w_own = (threadIdx.x % kDigitParts) * (kSortWarps / kDigitParts);
    for (int shift = shift0; shift < shift_end; shift += 8) {
        for (int d = lane; d < 256; d += 32) cnt[d] = 0;
        __syncwarp();
        // rounds of 32 keys, the keys of kRounds rounds loaded at once (in global memory each
        // round would otherwise wait for its own load)
        for (int base0 = lo; base0 < hi; base0 += kRounds * 32) {
            unsigned long long kk[kRounds];
#pragma unroll
            for (int u = 0; u < kRounds; ++u) {
                const int e = base0 + 32 * u + lane;
                kk[u] = e < hi ? a[e] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < kRounds; ++u) {
                const int base = base0 + 32 * u;
                if (base >= hi) break;  // warp-uniform
                const int e = base + lane;
                const bool ok = e < hi;
                const unsigned act = __ballot_sync(0xffffffffu, ok);
                unsigned d = 0, peers = 0, before = 0;
                if (ok) {
                    d = (unsigned)(kk[u] >> shift) & 255u;
                    peers = digit_peers(act, d);
                    before = cnt[d];
                    if (kCacheRanks) s_rank[e] = (unsigned short)(before + __popc(peers & lt_mask));
                }
                __syncwarp();
                if (ok && (peers & lt_mask) == 0) cnt[d] = before + __popc(peers);
                __syncwarp();
            }
        }
        __syncthreads();
        // the scatter base of (digit d, warp w) is the count of all (digit, warp) pairs before it
        // in digit-major order: an exclusive scan over the CTA's threads, which are ordered the
        // same way, of each thread's sum over its warps, plus the running sum within them
        {
            unsigned run = 0;
#pragma unroll
            for (int w = w_own; w < w_own + kSortWarps / kDigitParts; ++w) {
                const unsigned c = s_cnt[w * 256 + d_own];
                s_cnt[w * 256 + d_own] = run;
                run += c;
            }
            unsigned x = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            unsigned off = x - run;
#pragma unroll
            for (int q = 0; q < kSortWarps; ++q) off += q < warp ? wsum[q] : 0u;
#pragma unroll
            for (int w = w_own; w < w_own + kSortWarps / kDigitParts; ++w) s_cnt[w * 256 + d_own] += off;
        }
        __syncthreads();
        if (kCacheRanks) {
            for (int e = lo + lane; e < hi; e += 32) {
                const unsigned long long k = a[e];
                b[cnt[(unsigned)(k >> shift) & 255u] + s_rank[e]] = k;
            }
        } else {
            for (int base0 = lo; base0 < hi; base0 += kRounds * 32) {
                unsigned long long kk[kRounds];
#pragma unroll
                for (int u = 0; u < kRounds; ++u) {
                    const int e = base0 + 32 * u + lane;
                    kk[u] = e < hi ? a[e] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < kRounds; ++u) {
                    const int base = base0 + 32 * u;
                    if (base >= hi) break;  // warp-uniform
                    const int e = base + lane;
                    const bool ok = e < hi;
                    const unsigned act = __ballot_sync(0xffffffffu, ok);
                    unsigned d = 0, peers = 0, pos = 0;
                    const unsigned long long k = kk[u];
                    if (ok) {
                        d = (unsigned)(k >> shift) & 255u;
                        peers = digit_peers(act, d);
                        pos = cnt[d] + __popc(peers & lt_mask);
                    }
                    __syncwarp();
                    if (ok) {
                        b[pos] = k;
                        if ((peers & lt_mask) == 0) cnt[d] += __popc(peers);
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        unsigned long long *t = a;
        a = b;
        b = t;
    }
    return a;
}

constexpr int kTieRun = 32;  // longest run of equal depths the tie pass orders by itself

constexpr int kBucketBits = 12;  // buckets of the one-pass shared-memory sort
constexpr int kBucketRun = 64;   // longest bucket the rank placement orders by itself
static_assert((1 << kBucketBits) + kSortWarps <= kSortWarps * 256 + kSortWarps, "bucket counts fit the count area");

// Sort of L <= kRadixCap compressed keys (depth - d0) << 32 | index in shared memory by the
// top kBucketBits bits of the db-bit depth spread, then each bucket by the full key: one
// shared-memory atomic per key gives its bucket and its slot in it, an exclusive scan of the
// bucket counts the bucket starts, a scatter puts every key in its bucket (in any order
// inside), and every key then counts the smaller keys of its bucket and moves to that rank
// (keys are distinct: the index differs). Buckets are short (L keys over 2^kBucketBits
// buckets), so the count costs little and is the same for every key of a bucket. A bucket
// longer than kBucketRun sets *s_long and the keys are returned grouped by bucket for the
// caller's fallback. Returns the buffer holding the result.
__device__ unsigned long long *bucket_sort(unsigned long long *a, unsigned long long *b, int L, unsigned d0, int db,
                                           unsigned *s_hist /* >= 2^kBucketBits + kSortWarps, zeroed */,
                                           unsigned short *s_rank, unsigned *s_long) {
    constexpr int NB = 1 << kBucketBits, PER = NB / kSortThreads;
    static_assert(NB % kSortThreads == 0, "whole buckets per thread");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bshift = max(0, db - kBucketBits);
    // the bucket of a key: the top kBucketBits bits of its depth above the segment's minimum
    auto bucket = [&](unsigned long long k) { return ((unsigned)(k >> 32) - d0) >> bshift; };
    unsigned *wsum = s_hist + NB;
    for (int e = tid; e < L; e += kSortThreads)
        s_rank[e] = (unsigned short)atomicAdd(&s_hist[bucket(a[e])], 1u);
    __syncthreads();
    {  // exclusive scan of the bucket counts; thread t owns buckets [t PER, (t+1) PER)
        unsigned v[PER], run = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            v[q] = run;
            run += s_hist[tid * PER + q];
        }
        unsigned x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        unsigned off = x - run;
#pragma unroll
        for (int q = 0; q < kSortWarps; ++q) off += q < warp ? wsum[q] : 0u;
#pragma unroll
        for (int q = 0; q < PER; ++q) s_hist[tid * PER + q] = off + v[q];
    }
    __syncthreads();
    for (int e = tid; e < L; e += kSortThreads) {
        const unsigned long long k = a[e];
        b[s_hist[bucket(k)] + s_rank[e]] = k;
    }
    __syncthreads();
    for (int p = tid; p < L; p += kSortThreads) {
        const unsigned long long k = b[p];
        const unsigned bk = bucket(k);
        const int lo = (int)s_hist[bk], hi = bk + 1 < (unsigned)NB ? (int)s_hist[bk + 1] : L;
        if (hi - lo > kBucketRun) {
            *s_long = 1u;
            continue;
        }
        int rank = 0;
        for (int q = lo; q < hi; ++q) rank += b[q] < k;
        a[lo + rank] = k;
    }
    __syncthreads();
    return *s_long ? b : a;  // b still holds every key for the fallback
}

// Sort of kRadixCap < L <= kMidCap keys held in shared memory as they are (a) by the same
// one-pass bucketing, but moving 2-byte positions instead of 8-byte keys so that half as many
// keys again fit in the same shared memory: a shared-memory atomic per
// key gives its bucket and its slot, a scan the bucket starts, each key's position goes to its
// bucket's run in s_pos, and every key counts the smaller keys of its bucket (read through the
// positions) and writes its Gaussian index straight to its rank in the tile's list `out`.
// Returns false when some bucket is longer than kBucketRun (its keys are then not written; the
// caller sorts the whole segment again another way).
__device__ bool bucket_sort_pos(const unsigned long long *a, int L, unsigned d0, int db,
                                unsigned *s_hist /* >= 2^kBucketBits + kSortWarps, zeroed */,
                                unsigned short *s_rank, unsigned short *s_pos, unsigned *s_long,
                                unsigned *__restrict__ out) {
    constexpr int NB = 1 << kBucketBits, PER = NB / kSortThreads;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bshift = max(0, db - kBucketBits);
    auto bucket = [&](unsigned long long k) { return ((unsigned)(k >> 32) - d0) >> bshift; };
    unsigned *wsum = s_hist + NB;
    for (int e = tid; e < L; e += kSortThreads)
        s_rank[e] = (unsigned short)atomicAdd(&s_hist[bucket(a[e])], 1u);
    __syncthreads();
    {  // exclusive scan of the bucket counts; thread t owns buckets [t PER, (t+1) PER)
        unsigned v[PER], run = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            v[q] = run;
            run += s_hist[tid * PER + q];
        }
        unsigned x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        unsigned off = x - run;
#pragma unroll
        for (int q = 0; q < kSortWarps; ++q) off += q < warp ? wsum[q] : 0u;
#pragma unroll
        for (int q = 0; q < PER; ++q) s_hist[tid * PER + q] = off + v[q];
    }
    __syncthreads();
    for (int e = tid; e < L; e += kSortThreads) s_pos[s_hist[bucket(a[e])] + s_rank[e]] = (unsigned short)e;
    __syncthreads();
    for (int p = tid; p < L; p += kSortThreads) {
        const unsigned long long k = a[s_pos[p]];
        const unsigned bk = bucket(k);
        const int lo = (int)s_hist[bk], hi = bk + 1 < (unsigned)NB ? (int)s_hist[bk + 1] : L;
        if (hi - lo > kBucketRun) {
            *s_long = 1u;
            continue;
        }
        int rank = 0;
        for (int q = lo; q < hi; ++q) rank += a[s_pos[q]] < k;
        out[lo + rank] = (unsigned)k;
    }
    __syncthreads();
    return *s_long == 0u;
}

// Persistent: CTAs take (frame, tile) segments from the LPT-ordered work list. A key is
// (depth, Gaussian index); it is compressed to (depth - min depth) << 32 | index. A segment of
// up to kRadixCap keys is sorted in shared memory by bucket_sort (one bucket pass, then each
// bucket by the full key), one of up to kMidCap keys by bucket_sort_pos (the same with 2-byte
// positions in place of moved keys). A longer one is radix-sorted in place in global memory
// (mostly L2) on the depth bits only, which leaves runs of equal depth in list order, and a tie
// pass orders each such run by index (insertion sort by the run's first thread). A bucket longer
// than kBucketRun or a run longer than kTieRun sends the segment to a full-key sort: radix passes
// on the index bits, then on the depth bits (a segment of bucket_sort_pos goes to the global-memory
// sort).
// The sort is bound by round trips to memory, so none of them waits on another: thread 0 claims
// work items three ahead and, one stage per item, loads the claimed item's tile id and then its
// list bounds while the CTA sorts the current segment; a segment that fits in shared memory
// arrives there by asynchronous copies, all in flight at once.
__global__ void __launch_bounds__(kSortThreads) k_tile_sort(Ctx c) {
    // [kRadixCap] x 2 keys, [kRadixCap] ranks, counts; the position sort uses the keys and ranks
    // area as [kMidCap] keys, [kMidCap] ranks, [kMidCap] positions
    extern __shared__ unsigned long long s_keys[];
    unsigned short *s_rank = reinterpret_cast<unsigned short *>(s_keys + 2 * kRadixCap);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(s_rank + kRadixCap);
    unsigned short *s_rank_mid = reinterpret_cast<unsigned short *>(s_keys + kMidCap);
    unsigned short *s_pos_mid = s_rank_mid + kMidCap;
    __shared__ unsigned s_cur, s_st, s_L, s_dmin, s_dmax, s_imax, s_long;
    pdl_enter();
    if (c.cnt->overflow) return;
    const unsigned n_work = c.cnt->n_work;
    // thread 0's pipeline: w1 / t1 the next item and its tile, w2 the item after it
    unsigned w1 = 0, t1 = 0, w2 = 0;
    if (threadIdx.x == 0) {
        const unsigned w0 = atomicAdd(&c.cnt->next_sort, 1u);
        w1 = atomicAdd(&c.cnt->next_sort, 1u);
        w2 = atomicAdd(&c.cnt->next_sort, 1u);
        const unsigned t0 = w0 < n_work ? c.work[w0] : 0u;
        t1 = w1 < n_work ? c.work[w1] : 0u;
        s_cur = w0 < n_work ? 1u : 0u;
        s_st = w0 < n_work ? c.tile_start[t0] : 0u;
        s_L = w0 < n_work ? c.tile_start[t0 + 1] - s_st : 0u;
        s_dmin = 0xffffffffu;
        s_dmax = 0u;
        s_imax = 0u;
        s_long = 0u;
    }
    __syncthreads();
    while (s_cur) {
        const unsigned st = s_st, L = s_L;
        unsigned nst = 0, nend = 0, t2 = 0, w3 = 0;
        if (threadIdx.x == 0) {  // consumed at the end of this segment and at the next one
            if (w1 < n_work) {
                nst = c.tile_start[t1];
                nend = c.tile_start[t1 + 1];
            }
            t2 = w2 < n_work ? c.work[w2] : 0u;
            w3 = atomicAdd(&c.cnt->next_sort, 1u);
        }
        const unsigned long long *g = c.keys + st;
        const bool in_smem = L <= (unsigned)kRadixCap;
        const bool mid = !in_smem && L <= (unsigned)kMidCap;  // the position bucket sort
        unsigned dmin = 0xffffffffu, dmax = 0u, imax = 0u;
        if (in_smem || mid) {
            for (unsigned e = threadIdx.x; e < L; e += blockDim.x) cp_async8(s_keys + e, g + e);
            for (int i = threadIdx.x; i < (1 << kBucketBits); i += blockDim.x) s_cnt[i] = 0u;  // bucket counts
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
        }
        for (unsigned e = threadIdx.x; e < L; e += blockDim.x) {
            const unsigned long long k = in_smem || mid ? s_keys[e] : g[e];
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
        const int ib = 32 - __clz(s_imax);       // bits of the largest index (0 if 0)
        const int db = 32 - __clz(s_dmax - d0);  // bits of the depth spread
        unsigned long long *a = in_smem ? s_keys : c.keys2 + st;
        unsigned long long *bb = in_smem ? s_keys + kRadixCap : c.keys + st;
        // the radix passes take keys compressed to (depth - d0) << 32 | index (the order is the
        // same); the bucket sort reads the keys as they are
        auto compress = [&](unsigned long long *dst, const unsigned long long *src) {
            for (unsigned e = threadIdx.x; e < L; e += blockDim.x) {
                const unsigned long long k = src[e];
                dst[e] = ((unsigned long long)((unsigned)(k >> 32) - d0) << 32) | (unsigned)k;
            }
            __syncthreads();
        };
        unsigned long long *res = nullptr;  // stays null when the keys' indices are already written
        bool done = false;
        if (mid) {
            done = bucket_sort_pos(s_keys, (int)L, d0, db, s_cnt, s_rank_mid, s_pos_mid, &s_long, c.sorted + st);
            __syncthreads();  // every thread has read the flag before it is cleared
            if (!done) {      // a crowded bucket: sort the segment in global memory below
                if (threadIdx.x == 0) s_long = 0u;
                __syncthreads();
            }
        }
        if (done) {
        } else if (in_smem) {
            res = bucket_sort(a, bb, (int)L, d0, db, s_cnt, s_rank, &s_long);
            if (s_long) {  // a bucket too crowded for the fix-up: the full key by radix passes
                compress(res, res);
                unsigned long long *other = res == a ? bb : a;
                res = radix_sort<true>(res, other, (int)L, 0, ib, s_cnt, s_rank);
                other = res == a ? bb : a;
                res = radix_sort<true>(res, other, (int)L, 32, 32 + db, s_cnt, s_rank);
            }
        } else {
            compress(a, g);
            res = radix_sort<false>(a, bb, (int)L, 32, 32 + db, s_cnt, nullptr);
            // ties: a run keeps its depth under any reordering, so run starts found by other
            // threads do not change while a run is being ordered
            for (unsigned e = threadIdx.x; e + 1 < L; e += blockDim.x) {
                const unsigned dep = (unsigned)(res[e] >> 32);
                if ((unsigned)(res[e + 1] >> 32) != dep || (e > 0 && (unsigned)(res[e - 1] >> 32) == dep))
                    continue;
                unsigned end = e + 2;
                while (end < L && end - e <= (unsigned)kTieRun && (unsigned)(res[end] >> 32) == dep) ++end;
                if (end - e > (unsigned)kTieRun) {
                    s_long = 1u;
                    continue;
                }
                for (unsigned i = e + 1; i < end; ++i) {
                    const unsigned long long k = res[i];
                    unsigned j = i;
                    for (; j > e && res[j - 1] > k; --j) res[j] = res[j - 1];
                    res[j] = k;
                }
            }
            __syncthreads();
            if (s_long) {
                unsigned long long *other = res == a ? bb : a;
                res = radix_sort<false>(res, other, (int)L, 0, ib, s_cnt, nullptr);
                other = res == a ? bb : a;
                res = radix_sort<false>(res, other, (int)L, 32, 32 + db, s_cnt, nullptr);
            }
        }
        if (res)
            for (unsigned e = threadIdx.x; e < L; e += blockDim.x) c.sorted[st + e] = (unsigned)res[e];
        __syncthreads();
        if (threadIdx.x == 0) {
            s_cur = w1 < n_work ? 1u : 0u;
            s_st = nst;
            s_L = nend - nst;
            w1 = w2;
            t1 = t2;
            w2 = w3;
            s_dmin = 0xffffffffu;
            s_dmax = 0u;
            s_imax = 0u;
            s_long = 0u;
        }
        __syncthreads();
    }
    // the last CTA out puts the work counter back to zero for the next launch
    if (threadIdx.x == 0 && atomicAdd(&c.cnt->done_sort, 1u) == gridDim.x - 1) {
        c.cnt->next_sort = 0u;
        c.cnt->done_sort = 0u;
    }
}

}  // namespace

cudaError_t launch_scan(const Ctx &c, cudaStream_t s) {
    const unsigned nb = (unsigned)((c.T + kScanTile - 1) / kScanTile);
    cudaError_t e = launch_pdl(k_scan_blocks, dim3(nb), dim3(kScanTile), 0, s, c);
    if (e != cudaSuccess) return e;
    if ((e = launch_pdl(k_scan_top, dim3(1), dim3(kScanTile), 0, s, c)) != cudaSuccess) return e;
    return launch_pdl(k_scan_write, dim3(nb), dim3(kScanTile), 0, s, c);
}

size_t scan_aux_bytes(long long T) {
    const long long nb = (T + kScanTile - 1) / kScanTile;
    return (size_t)nb * 8 + (size_t)nb * 4 + (size_t)nb * 32 * 4 + 32 * 4;
}

cudaError_t launch_scatter(const Ctx &c, int max_n, cudaStream_t s) {
    if (c.B == 0 || max_n == 0) return cudaSuccess;
    dim3 grid((max_n + kScatterThreads - 1) / kScatterThreads, c.B);
    return launch_pdl(k_scatter, grid, dim3(kScatterThreads), 0, s, c);
}

cudaError_t launch_tile_sort(const Ctx &c, int sms, cudaStream_t s) {
    static int attr_device = -1, per_sm = 1;
    const int smem = 2 * kRadixCap * (int)sizeof(unsigned long long) + kRadixCap * (int)sizeof(unsigned short) +
                     (kSortWarps * 256 + kSortWarps) * 4;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_device != dev) {
        e = cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_sort, kSortThreads, smem);
        if (e != cudaSuccess) return e;
        per_sm = per_sm < 1 ? 1 : per_sm;
        attr_device = dev;
    }
    return launch_pdl(k_tile_sort, dim3(sms * per_sm), dim3(kSortThreads), (size_t)smem, s, c);
}

}  // namespace rgba
