// Frontier selection for Residual BP and Residual Splash (Section III-A):
// exact top-k by residual with ties to the smaller id, one thread-block
// cluster per graph.
//
// The paper sorts (key-value radix sort) and takes the prefix. Here each graph
// is owned by a cluster of C CTAs (C chosen so the grid covers the SMs); every
// CTA stages a contiguous slice of the graph's keys (the residual's IEEE bits:
// non-negative floats order as unsigned integers) in shared memory. An MSB
// radix select narrows the k-th largest key one byte per pass: each CTA builds
// a 256-bin histogram of its slice, the CTAs sum the cluster's histograms
// through distributed shared memory, and every CTA takes the same digit
// decision. An ordered pass then takes every key above the threshold and the
// lowest-id ties (ranked across the cluster when ties straddle the threshold).
// RBP commits the selected messages in that pass; RS marks its splash roots.
#include "bp_internal.cuh"
#include "bp_launch.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace bpg {

constexpr int SEL_THREADS = 1024;
// Keys of a CTA's slice are staged in dynamic shared memory when they fit.
constexpr int SEL_SMEM_BYTES = 200 * 1024;

__device__ __forceinline__ uint32_t key_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long key_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v);
}

// Shared state of the cluster-wide selection (one instance per CTA).
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

// Cluster-wide threshold: thr = k-th largest key over the union of the CTAs'
// slices (1 <= k <= total count), take_eq = keys equal to thr inside the top
// k, eq_total = keys equal to thr. Every thread of every CTA of the cluster
// must call it.
template <typename KeyT, typename KeyFn>
__device__ void cluster_select_threshold(cg::cluster_group &cl, SelShared<KeyT> &sh, int n_local, int k,
                                         KeyFn key, KeyT &thr, int &take_eq, int &eq_total)
{
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

// RBP: select the top k_sel messages of each running graph and commit them.
template <typename S>
__global__ void __launch_bounds__(SEL_THREADS) k_select_rbp(DevGraph g, DevRun dr, RunParams rp)
{
    using RT = typename ResidT<S>::T;
    using KeyT = decltype(key_bits((RT)0));
    __shared__ SelShared<KeyT> sh;
    extern __shared__ __align__(16) unsigned char sel_smem[];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned C = cl.num_blocks(), rank = cl.block_rank();
    const int gg = blockIdx.x / C;
    const GState st = dr.gs[gg];   // the same for every CTA of the cluster
    if (st.status != ST_RUNNING)
        return;
    const int e0 = g.ge_off[gg];
    const int cnt = g.ge_off[gg + 1] - e0;
    if (cnt == 0)
        return;
    int lo, hi;
    slice_of(cnt, rank, C, lo, hi);
    const int nl = hi - lo;
    const RT *R = (const RT *)dr.resid + e0 + lo;
    KeyT *s_keys = reinterpret_cast<KeyT *>(sel_smem);
    const bool staged = (size_t)nl * sizeof(KeyT) <= (size_t)g.sel_smem_bytes;
    if (staged)
        stage_keys<KeyT>(nl, s_keys, [&](int idx) { return key_bits(R[idx]); });
    auto key = [&](int idx) -> KeyT { return staged ? s_keys[idx] : key_bits(R[idx]); };
    KeyT thr;
    int take_eq, eq_total;
    cluster_select_threshold<KeyT>(cl, sh, nl, st.k_sel, key, thr, take_eq, eq_total);
    S *dst = (S *)dr.msg[0];
    const S *src = (const S *)dr.msg[1];
    const int epm = g.epm;
    const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
    cluster_select_apply<KeyT>(cl, sh, nl, thr, take_eq, eq_total, key, [&](int idx, bool take) {
        if (!take)
            return;
        const int e = e0 + lo + idx;
        for (int x = 0; x < epm; ++x)
            dst[(size_t)e * epm + x] = src[(size_t)e * epm + x];
        if (tr)
            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (e >> 5)], 1u << (e & 31));
    });
}

// RS: vertex residual = max residual of the messages into the vertex; select
// the top k_sel vertices as splash roots (level 0), every other vertex gets
// level -1. Each CTA owns a slice of the graph's vertices.
template <typename S>
__global__ void __launch_bounds__(SEL_THREADS) k_select_rs(DevGraph g, DevRun dr, RunParams rp)
{
    using RT = typename ResidT<S>::T;
    using KeyT = decltype(key_bits((RT)0));
    __shared__ SelShared<KeyT> sh;
    extern __shared__ __align__(16) unsigned char sel_smem[];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned C = cl.num_blocks(), rank = cl.block_rank();
    const int gg = blockIdx.x / C;
    const GState st = dr.gs[gg];
    if (st.status != ST_RUNNING)
        return;
    const int v0 = g.gv_off[gg];
    const int nv = g.gv_off[gg + 1] - v0;
    if (nv == 0)
        return;
    int lo, hi;
    slice_of(nv, rank, C, lo, hi);
    const int per = (nv + (int)C - 1) / (int)C;
    const int nl = hi - lo;
    // every CTA uses shared memory for its slice when the largest slice fits,
    // else the global vertex-residual array. Pull form: vertex v gathers the
    // residuals of its incoming messages R[rev[f]], f in row v (four vertices
    // per thread in flight).
    const bool staged = (size_t)per * sizeof(KeyT) <= (size_t)g.sel_smem_bytes;
    KeyT *vkeys = staged ? reinterpret_cast<KeyT *>(sel_smem) : reinterpret_cast<KeyT *>(dr.vres) + v0 + lo;
    const RT *R = (const RT *)dr.resid;
    constexpr int U = 4;
    for (int base = threadIdx.x; base < nl; base += U * blockDim.x) {
        int rb[U], re[U];
        RT m[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            m[u] = 0;
            rb[u] = re[u] = 0;
            if (idx < nl) {
                rb[u] = g.row_ptr[v0 + lo + idx];
                re[u] = g.row_ptr[v0 + lo + idx + 1];
            }
        }
        for (int j = 0;; ++j) {
            bool any = false;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (rb[u] + j < re[u]) {
                    const RT r = R[g.rev[rb[u] + j]];
                    m[u] = r > m[u] ? r : m[u];
                    any = true;
                }
            }
            if (!any)
                break;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = base + u * blockDim.x;
            if (idx < nl)
                vkeys[idx] = key_bits(m[u]);
        }
    }
    __syncthreads();
    auto key = [&](int idx) -> KeyT { return vkeys[idx]; };
    KeyT thr;
    int take_eq, eq_total;
    cluster_select_threshold<KeyT>(cl, sh, nl, st.k_sel, key, thr, take_eq, eq_total);
    const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
    cluster_select_apply<KeyT>(cl, sh, nl, thr, take_eq, eq_total, key, [&](int idx, bool take) {
        const int v = v0 + lo + idx;
        dr.level[v] = take ? (int8_t)0 : (int8_t)-1;
        if (take && tr)
            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (v >> 5)], 1u << (v & 31));
    });
    cl.sync();   // no CTA leaves while a peer may still address its shared memory
}

template <typename K> static void set_smem_attr(K kernel)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SEL_SMEM_BYTES);
}

void prepare_select_kernels()
{
    set_smem_attr(k_select_rbp<double>);
    set_smem_attr(k_select_rbp<float>);
    set_smem_attr(k_select_rbp<__nv_bfloat16>);
    set_smem_attr(k_select_rbp<int16_t>);
    set_smem_attr(k_select_rs<double>);
    set_smem_attr(k_select_rs<float>);
}

int select_smem_limit() { return SEL_SMEM_BYTES; }

// CTAs per graph: enough clusters to cover the SMs, at most 8 (portable size).
static unsigned cluster_size(int G)
{
    int c = 152 / (G > 0 ? G : 1);
    c = c < 1 ? 1 : (c > 8 ? 8 : c);
    return (unsigned)c;
}

template <typename K>
static void launch_clustered(K kernel, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    const unsigned C = cluster_size(g.G);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.G * C, 1, 1);
    cfg.blockDim = dim3(SEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)g.sel_smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, g, dr, rp);
}

void launch_select_rbp(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    switch (dtype) {
    case DT_F64: launch_clustered(k_select_rbp<double>, g, dr, rp, s); break;
    case DT_F32: launch_clustered(k_select_rbp<float>, g, dr, rp, s); break;
    case DT_BF16: launch_clustered(k_select_rbp<__nv_bfloat16>, g, dr, rp, s); break;
    default: launch_clustered(k_select_rbp<int16_t>, g, dr, rp, s); break;
    }
}

void launch_select_rs(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    // selection reads residuals only: FP64 runs keep double residuals, the others float
    if (dtype == DT_F64)
        launch_clustered(k_select_rs<double>, g, dr, rp, s);
    else
        launch_clustered(k_select_rs<float>, g, dr, rp, s);
}

}  // namespace bpg
