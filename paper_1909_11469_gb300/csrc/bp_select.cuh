// Cluster-wide exact top-k selection (device functions shared by the
// per-round selection kernels and the persistent batch kernel).
//
// Every CTA of a cluster owns a contiguous slice of a graph's keys (the
// residual's IEEE bits: non-negative floats order as unsigned integers). An
// MSB radix select narrows the k-th largest key one digit per pass: each CTA
// builds a histogram of its slice, the CTAs sum the cluster's histograms
// through distributed shared memory, and every CTA takes the same digit
// decision. 32-bit keys take three passes (11, 11 and 10 bits) with one
// histogram array per pass, so a pass never clears an array a peer may still
// read and one cluster barrier per pass suffices; the keys that survive the
// second pass are compacted, so the third pass touches only them. 64-bit keys
// take eight 8-bit passes. An ordered pass takes every key above the threshold
// and the lowest-id ties, ranked across the cluster when ties straddle it.
#pragma once

#include "bp_internal.cuh"

#include <cooperative_groups.h>

namespace bpg {

namespace cg = cooperative_groups;

constexpr int SEL_THREADS = 1024;
// Keys of a CTA's slice are staged in dynamic shared memory when they fit.
constexpr int SEL_SMEM_BYTES = 176 * 1024;
// Candidates of the third pass of the 32-bit select held per CTA.
constexpr int SEL_CAND = 4096;

__device__ __forceinline__ uint32_t key_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long key_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v);
}

// Shared state of the cluster-wide selection (one instance per CTA); 64-bit keys.
template <typename KeyT> struct SelShared {
    unsigned int hist[256];
    unsigned int total[256];
    KeyT prefix;
    int krem;
    int bucket;
    unsigned int warp_cnt[32];
    int eq_before;    // keys equal to thr in lower-ranked CTAs of the cluster
    int taken;        // running rank among ties inside this CTA
    int my_eq;        // keys equal to thr in this CTA's slice
};

// 32-bit keys: one histogram per pass and the compacted candidates.
template <> struct SelShared<uint32_t> {
    unsigned int hist1[2048];   // key bits 31..21
    unsigned int hist2[2048];   // key bits 20..10 (keys whose bits 31..21 match)
    unsigned int hist3[1024];   // key bits 9..0 (keys whose bits 31..10 match)
    uint32_t cand[SEL_CAND];    // this CTA's keys that match bits 31..21 (when they fit)
    int n_cand;
    uint32_t prefix;
    int krem;
    int bucket;
    unsigned int warp_cnt[32];
    unsigned int warp_scan[32];
    int eq_before;
    int taken;
    int my_eq;
};

// Adds one key digit per lane to a shared histogram (d = 0xffffffff: none):
// one shared atomic per distinct digit per warp (residuals cluster in a few
// exponent bins, so per-lane atomics would serialise). Whole warps only.
__device__ __forceinline__ void hist_add(unsigned int *hist, unsigned d)
{
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (d != 0xffffffffu && (threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(&hist[d], (unsigned)__popc(peers));
}

// Sums the cluster's copies of a NB-bin histogram (after a cluster barrier)
// and finds the digit that holds the krem-th largest key: thread t owns the
// NB / SEL_THREADS bins starting at the t-th from the top (blocks of
// SEL_THREADS threads), a block-wide scan of
// the owned sums locates the digit. Every CTA computes the same result, into
// sh.prefix (digit), sh.krem (rank inside the digit) and sh.bucket (its
// cluster-wide count).
template <int NB>
__device__ __forceinline__ void cluster_digit(cg::cluster_group &cl, SelShared<uint32_t> &sh, unsigned int *hist,
                                              int krem)
{
    const unsigned C = cl.num_blocks();
    constexpr int per = NB / SEL_THREADS;   // bins per thread; blocks of SEL_THREADS threads
    unsigned v[per];
    unsigned mine = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        const int d = NB - 1 - ((int)threadIdx.x * per + q);
        unsigned s = 0;
        for (unsigned r = 0; r < C; ++r)
            s += cl.map_shared_rank(hist, r)[d];
        v[q] = s;
        mine += s;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        sh.warp_cnt[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        unsigned w = lane < nw ? sh.warp_cnt[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += y;
        }
        sh.warp_scan[lane] = wi - w;   // exclusive
    }
    __syncthreads();
    incl += sh.warp_scan[warp];
    unsigned acc = incl - mine;
    if (acc < (unsigned)krem && (unsigned)krem <= incl) {
        // the digit is among this thread's bins, walked from the top
#pragma unroll
        for (int q = 0; q < per; ++q) {
            if (acc + v[q] >= (unsigned)krem) {
                sh.prefix = (uint32_t)(NB - 1 - ((int)threadIdx.x * per + q));
                sh.krem = krem - (int)acc;
                sh.bucket = (int)v[q];
                break;
            }
            acc += v[q];
        }
    }
    __syncthreads();
}

// Clears the histograms and the candidate count of the 32-bit select (every
// thread of the CTA calls it; a __syncthreads must follow).
__device__ __forceinline__ void sel32_clear(SelShared<uint32_t> &sh)
{
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
        sh.hist1[t] = 0u;
        sh.hist2[t] = 0u;
    }
    for (int t = threadIdx.x; t < 1024; t += blockDim.x)
        sh.hist3[t] = 0u;
    if (threadIdx.x == 0)
        sh.n_cand = 0;
}

// Pass-1 digit (key bits 31..21) of a 32-bit key; 0xffffffff = no key.
__device__ __forceinline__ unsigned sel32_digit1(uint32_t key) { return key >> 21; }

// 32-bit cluster-wide threshold (see cluster_select_threshold). pass1_done:
// the caller has cleared the histograms (sel32_clear) and already added every
// key's pass-1 digit to sh.hist1 (while staging the keys).
template <typename KeyFn>
__device__ void cluster_select_threshold32(cg::cluster_group &cl, SelShared<uint32_t> &sh, int n_local, int k,
                                           KeyFn key, uint32_t &thr, int &take_eq, int &eq_total,
                                           bool pass1_done)
{
    if (!pass1_done) {
        sel32_clear(sh);
        __syncthreads();
        // pass 1: bits 31..21
        for (int base = 0; base < n_local; base += blockDim.x) {
            const int idx = base + threadIdx.x;
            hist_add(sh.hist1, idx < n_local ? sel32_digit1(key(idx)) : 0xffffffffu);
        }
    }
    cl.sync();   // every CTA's first histogram is complete
    cluster_digit<2048>(cl, sh, sh.hist1, k);
    const uint32_t d1 = sh.prefix;
    int krem = sh.krem;
    // pass 2: bits 20..10 of the keys in digit d1; they are also compacted
    // when this CTA's share fits
    const bool compact = sh.hist1[d1] <= (unsigned)SEL_CAND;
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < n_local; base += blockDim.x) {
        const int idx = base + threadIdx.x;
        const uint32_t kv = idx < n_local ? key(idx) : 0u;
        const bool in = idx < n_local && (kv >> 21) == d1;
        hist_add(sh.hist2, in ? (kv >> 10) & 2047u : 0xffffffffu);
        if (compact) {
            const unsigned b = __ballot_sync(0xffffffffu, in);
            int pos = 0;
            if (lane == 0 && b)
                pos = atomicAdd(&sh.n_cand, __popc(b));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (in)
                sh.cand[pos + __popc(b & ((1u << lane) - 1u))] = kv;
        }
    }
    cl.sync();
    cluster_digit<2048>(cl, sh, sh.hist2, krem);
    const uint32_t pre2 = (d1 << 11) | sh.prefix;
    krem = sh.krem;
    // pass 3: bits 9..0 of the keys that match bits 31..10
    const int nc = compact ? sh.n_cand : n_local;
    for (int base = 0; base < nc; base += blockDim.x) {
        const int idx = base + threadIdx.x;
        unsigned d = 0xffffffffu;
        if (idx < nc) {
            const uint32_t kv = compact ? sh.cand[idx] : key(idx);
            if ((kv >> 10) == pre2)
                d = kv & 1023u;
        }
        hist_add(sh.hist3, d);
    }
    cl.sync();
    cluster_digit<1024>(cl, sh, sh.hist3, krem);
    // no CTA may leave (or reuse its histograms) while a peer still reads them
    cl.sync();
    thr = (pre2 << 10) | sh.prefix;
    take_eq = sh.krem;
    eq_total = sh.bucket;
}

// Cluster-wide threshold: thr = k-th largest key over the union of the CTAs'
// slices (1 <= k <= total count), take_eq = keys equal to thr inside the top
// k, eq_total = keys equal to thr. Every thread of every CTA of the cluster
// must call it.
template <typename KeyT, typename KeyFn>
__device__ void cluster_select_threshold(cg::cluster_group &cl, SelShared<KeyT> &sh, int n_local, int k,
                                         KeyFn key, KeyT &thr, int &take_eq, int &eq_total,
                                         bool pass1_done = false)
{
    if constexpr (sizeof(KeyT) == 4) {
        cluster_select_threshold32(cl, sh, n_local, k, key, thr, take_eq, eq_total, pass1_done);
        return;
    } else {
    const unsigned C = cl.num_blocks();
    KeyT prefix = 0, mask = 0;
    int krem = k;
    for (int pass = 0; pass < (int)sizeof(KeyT); ++pass) {
        const int shift = ((int)sizeof(KeyT) - 1 - pass) * 8;
        for (int t = threadIdx.x; t < 256; t += blockDim.x)
            sh.hist[t] = 0u;
        __syncthreads();
        // one shared atomic per distinct digit per warp (residuals cluster in a
        // few exponent bins, so per-thread atomics would serialise)
        for (int base = 0; base < n_local; base += blockDim.x) {
            const int idx = base + threadIdx.x;
            unsigned d = 0xffffffffu;
            if (idx < n_local) {
                const KeyT kv = key(idx);
                if ((kv & mask) == prefix)
                    d = (unsigned)((kv >> shift) & (KeyT)255);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (d != 0xffffffffu && (threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(&sh.hist[d], (unsigned)__popc(peers));
        }
        cl.sync();   // every CTA's histogram is complete
        for (int t = threadIdx.x; t < 256; t += blockDim.x) {
            unsigned s = 0;
            for (unsigned r = 0; r < C; ++r)
                s += cl.map_shared_rank(&sh.hist[0], r)[t];
            sh.total[t] = s;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane L owns digits 255-8L down to 248-8L (descending order)
            const int lane = threadIdx.x;
            unsigned loc[8];
            unsigned sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                loc[q] = sh.total[255 - 8 * lane - q];
                sum += loc[q];
            }
            unsigned incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            const unsigned excl = incl - sum;
            if (excl < (unsigned)krem && (unsigned)krem <= incl) {
                unsigned acc = excl;
                int d = 255 - 8 * lane - 7;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (acc + loc[q] >= (unsigned)krem) {
                        d = 255 - 8 * lane - q;
                        break;
                    }
                    acc += loc[q];
                }
                sh.prefix = prefix | ((KeyT)d << shift);
                sh.krem = krem - (int)acc;
                sh.bucket = (int)sh.total[d];
            }
        }
        cl.sync();   // nobody clears its histogram while another CTA still reads it
        prefix = sh.prefix;
        krem = sh.krem;
        mask |= ((KeyT)255 << shift);
    }
    thr = prefix;
    take_eq = krem;
    eq_total = sh.bucket;
    }
}

// Ordered pass over this CTA's slice: on_item(idx, take) for every local idx,
// take = key above thr, or equal to thr and among the first take_eq such keys
// of the cluster in global index order (CTA rank order, then local order).
template <typename KeyT, typename KeyFn, typename ItemFn>
__device__ void cluster_select_apply(cg::cluster_group &cl, SelShared<KeyT> &sh, int n_local, KeyT thr,
                                     int take_eq, int eq_total, KeyFn key, ItemFn on_item)
{
    if (take_eq == eq_total) {
        // every key equal to thr is in the top k: no ranking of ties needed
        for (int idx = threadIdx.x; idx < n_local; idx += blockDim.x)
            on_item(idx, key(idx) >= thr);
        return;
    }
    // ties straddle the threshold: rank them across the cluster
    if (threadIdx.x == 0)
        sh.my_eq = 0;
    __syncthreads();
    int mine = 0;
    for (int idx = threadIdx.x; idx < n_local; idx += blockDim.x)
        mine += key(idx) == thr;
    if (mine)
        atomicAdd(&sh.my_eq, mine);
    cl.sync();
    if (threadIdx.x == 0) {
        int before = 0;
        for (unsigned r = 0; r < cl.block_rank(); ++r)
            before += *cl.map_shared_rank(&sh.my_eq, r);
        sh.eq_before = before;
        sh.taken = 0;
    }
    cl.sync();   // keep my_eq readable until every CTA has summed it
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < n_local; base += blockDim.x) {
        const int idx = base + threadIdx.x;
        const bool in = idx < n_local;
        const KeyT kv = in ? key(idx) : (KeyT)0;
        const bool gt = in && kv > thr;
        const bool eq = in && kv == thr;
        const unsigned b = __ballot_sync(0xffffffffu, eq);
        if (lane == 0)
            sh.warp_cnt[warp] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w)
            before += (int)sh.warp_cnt[w];
        const int rank = sh.eq_before + sh.taken + before + __popc(b & ((1u << lane) - 1u));
        if (in)
            on_item(idx, gt || (eq && rank < take_eq));
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nw; ++w)
                tot += (int)sh.warp_cnt[w];
            sh.taken += tot;
        }
        __syncthreads();
    }
}

// Copies n keys into shared memory (eight independent loads in flight per
// thread) and adds each key's pass-1 digit to hist (whole warps: the loop
// bounds are the same for every thread).
template <typename LoadFn>
__device__ void stage_keys_hist(int n, uint32_t *s_keys, LoadFn load, unsigned int *hist)
{
    constexpr int U = 8;
    for (int b0 = 0; b0 < n; b0 += U * blockDim.x) {
        uint32_t v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = b0 + threadIdx.x + u * blockDim.x;
            if (idx < n)
                v[u] = load(idx);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = b0 + threadIdx.x + u * blockDim.x;
            if (idx < n)
                s_keys[idx] = v[u];
            hist_add(hist, idx < n ? sel32_digit1(v[u]) : 0xffffffffu);
        }
    }
    __syncthreads();
}

// Copies n keys into shared memory with eight independent loads in flight per
// thread.
template <typename KeyT, typename LoadFn>
__device__ void stage_keys(int n, KeyT *s_keys, LoadFn load)
{
    constexpr int U = 8;
    for (int base = threadIdx.x; base < n; base += U * blockDim.x) {
        KeyT v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < n)
                v[u] = load(idx);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < n)
                s_keys[idx] = v[u];
        }
    }
    __syncthreads();
}

// Slice [lo, hi) of count items owned by CTA rank r of C.
__device__ __forceinline__ void slice_of(int count, unsigned r, unsigned C, int &lo, int &hi)
{
    const int per = (count + (int)C - 1) / (int)C;
    lo = min(count, (int)r * per);
    hi = min(count, lo + per);
}

}  // namespace bpg
