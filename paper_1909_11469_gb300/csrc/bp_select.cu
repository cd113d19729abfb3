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
#include "bp_select.cuh"

namespace bpg {

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
