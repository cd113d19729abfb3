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
#include "bp_update.cuh"

#include <algorithm>
#include <cmath>

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
    bool pass1 = false;
    if constexpr (sizeof(KeyT) == 4) {
        if (staged) {
            // the first radix pass rides on the staging loop
            sel32_clear(sh);
            __syncthreads();
            stage_keys_hist(nl, s_keys, [&](int idx) { return key_bits(R[idx]); }, sh.hist1);
            pass1 = true;
        }
    }
    if (staged && !pass1)
        stage_keys<KeyT>(nl, s_keys, [&](int idx) { return key_bits(R[idx]); });
    auto key = [&](int idx) -> KeyT { return staged ? s_keys[idx] : key_bits(R[idx]); };
    KeyT thr;
    int take_eq, eq_total;
    cluster_select_threshold<KeyT>(cl, sh, nl, st.k_sel, key, thr, take_eq, eq_total, pass1);
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
// level -1, then the BFS levels 1..h and (binary messages) the per-level
// vertex lists of the sweeps, one list per level for the whole batch. Each
// CTA owns a slice of the graph's vertices.
template <typename S>
__global__ void __launch_bounds__(SEL_THREADS, 2) k_select_rs(DevGraph g, DevRun dr, RunParams rp)
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
    // 32-bit keys: the first radix pass rides on this loop (uniform bounds:
    // every warp calls hist_add with all lanes)
    constexpr bool fuse1 = sizeof(KeyT) == 4;
    if constexpr (fuse1) {
        sel32_clear(sh);
        __syncthreads();
    }
    for (int b0 = 0; b0 < nl; b0 += U * blockDim.x) {
        const int base = b0 + (int)threadIdx.x;
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
            if constexpr (fuse1)
                hist_add(sh.hist1, idx < nl ? sel32_digit1(key_bits(m[u])) : 0xffffffffu);
        }
    }
    __syncthreads();
    auto key = [&](int idx) -> KeyT { return vkeys[idx]; };
    KeyT thr;
    int take_eq, eq_total;
    cluster_select_threshold<KeyT>(cl, sh, nl, st.k_sel, key, thr, take_eq, eq_total, fuse1);
    const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
    cluster_select_apply<KeyT>(cl, sh, nl, thr, take_eq, eq_total, key, [&](int idx, bool take) {
        const int v = v0 + lo + idx;
        dr.level[v] = take ? (int8_t)0 : (int8_t)-1;
        if (take && tr)
            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (v >> 5)], 1u << (v & 31));
    });
    // The cluster owns the whole graph, so the splash levels 1..h (multi-source
    // BFS, pull form) are formed here too, a cluster barrier between levels.
    // Each vertex's level is written only by the thread that owns it.
    const int h = rp.splash_depth;
    for (int d = 1; d <= h; ++d) {
        cl.sync();   // level d - 1 of every slice is visible
        for (int idx = threadIdx.x; idx < nl; idx += blockDim.x)
            bfs_vertex(g, dr, v0 + lo + idx, d);
    }
    if (dr.lvl_list && h <= LVL_MAX && g.epm == 1) {
        // per-level vertex lists of the sweeps (one reservation per level per
        // CTA) and the round's sweep counts: a level-0 vertex is evaluated and
        // committed once, a deeper one twice
        __shared__ int s_cnt[LVL_MAX + 1];
        __shared__ int s_base[LVL_MAX + 1];
        __shared__ unsigned long long s_commit;
        if (threadIdx.x <= (unsigned)LVL_MAX)
            s_cnt[threadIdx.x] = 0;
        if (threadIdx.x == 0)
            s_commit = 0ull;
        __syncthreads();
        const unsigned lane = threadIdx.x & 31;
        // counts per level (one shared atomic per warp and level)
        for (int base = 0; base < nl; base += blockDim.x) {
            const int idx = base + threadIdx.x;
            const int lv = idx < nl ? (int)dr.level[v0 + lo + idx] : -1;
            for (int L = 0; L <= h; ++L) {
                const unsigned m = __ballot_sync(0xffffffffu, lv == L);
                if (lane == 0 && m)
                    atomicAdd(&s_cnt[L], __popc(m));
            }
        }
        __syncthreads();
        if (threadIdx.x <= (unsigned)h) {
            const int c = s_cnt[threadIdx.x];
            int b = 0;
            if (c)
                b = atomicAdd(&dr.lvl_cnt[threadIdx.x], c);
            s_base[threadIdx.x] = b;
            s_cnt[threadIdx.x] = 0;
        }
        __syncthreads();
        unsigned long long c = 0;
        for (int base = 0; base < nl; base += blockDim.x) {
            const int idx = base + threadIdx.x;
            const int v = v0 + lo + idx;
            const int lv = idx < nl ? (int)dr.level[v] : -1;
            for (int L = 0; L <= h; ++L) {
                const unsigned m = __ballot_sync(0xffffffffu, lv == L);
                int wpos = 0;
                if (lane == 0 && m)
                    wpos = atomicAdd(&s_cnt[L], __popc(m));
                wpos = __shfl_sync(0xffffffffu, wpos, 0);
                if (lv == L) {
                    const int beg = g.row_ptr[v];
                    dr.lvl_list[(size_t)L * g.n + s_base[L] + wpos +
                                __popc(m & ((1u << lane) - 1u))] = make_int2(v, beg);
                    c += (unsigned long long)(g.row_ptr[v + 1] - beg) * (L == 0 ? 1u : 2u);
                }
            }
        }
        c += __shfl_xor_sync(0xffffffffu, c, 16);
        c += __shfl_xor_sync(0xffffffffu, c, 8);
        c += __shfl_xor_sync(0xffffffffu, c, 4);
        c += __shfl_xor_sync(0xffffffffu, c, 2);
        c += __shfl_xor_sync(0xffffffffu, c, 1);
        if (lane == 0 && c)
            atomicAdd(&s_commit, c);
        __syncthreads();
        if (threadIdx.x == 0 && s_commit) {
            atomicAdd(&dr.gs[gg].committed, s_commit);
            atomicAdd(&dr.gs[gg].evals, s_commit);
        }
    }
    cl.sync();   // no CTA leaves while a peer may still address its shared memory
}

template <typename K> static void set_smem_attr(K kernel)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SEL_SMEM_BYTES);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
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

// Cluster shape of one selection kernel over G graphs of at most max_keys
// keys: every cluster owns one graph and every CTA a slice of it, staged in
// shared memory. For each cluster size c = 1..8 the occupancy query gives how
// many clusters fit on the GPU at once (clusters are placed inside one GPC, so
// this is below 152 / c); the shape with the least estimated time wins, where
// a wave of clusters costs a fixed ~12 us (passes, barriers) plus ~1 us per
// 1000 keys of a slice.
template <typename K>
static double plan_one(K kernel, int G, int max_keys, int key_bytes, int32_t &c_out, int32_t &dyn_out)
{
    double best = 1e300;
    c_out = 1;
    dyn_out = 0;
    for (int c = 1; c <= 8; ++c) {
        const long long per = ((long long)max_keys + c - 1) / c;
        long long bytes = (per * key_bytes + 15) / 16 * 16;
        if (bytes > SEL_SMEM_BYTES)
            bytes = SEL_SMEM_BYTES;   // larger slices read their keys from global memory
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(c * std::max(1, std::min(G, 64))), 1, 1);
        cfg.blockDim = dim3(SEL_THREADS, 1, 1);
        cfg.dynamicSmemBytes = (size_t)bytes;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, kernel, &cfg) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            continue;
        }
        const double waves = (double)((G + ncl - 1) / ncl);
        const double cost = waves * (12.0 + (double)per / 1000.0);
        if (cost < best) {
            best = cost;
            c_out = c;
            dyn_out = (int32_t)bytes;
        }
    }
    return best;
}


// Estimated time of the grid-wide selection: ~6 us per kernel (measured: 50
// graphs of 39,600 keys took ~70 us in 10 kernels) plus every key of every
// graph at ~150,000 keys per us over the whole GPU.
static double grid_cost(int dtype, bool rs, int G, int max_keys)
{
    return 6.0 * grid_select_launches(dtype, rs) + (double)G * (double)max_keys / 150000.0;
}

void plan_select(int dtype, int G, int max_ge, int max_gv, int32_t c_out[2], int32_t dyn_out[2],
                 int32_t grid_out[2])
{
    double t_rbp, t_rs;
    switch (dtype) {
    case DT_F64: t_rbp = plan_one(k_select_rbp<double>, G, max_ge, 8, c_out[0], dyn_out[0]); break;
    case DT_F32: t_rbp = plan_one(k_select_rbp<float>, G, max_ge, 4, c_out[0], dyn_out[0]); break;
    case DT_BF16: t_rbp = plan_one(k_select_rbp<__nv_bfloat16>, G, max_ge, 4, c_out[0], dyn_out[0]); break;
    default: t_rbp = plan_one(k_select_rbp<int16_t>, G, max_ge, 4, c_out[0], dyn_out[0]); break;
    }
    if (dtype == DT_F64)
        t_rs = plan_one(k_select_rs<double>, G, max_gv, 8, c_out[1], dyn_out[1]);
    else
        t_rs = plan_one(k_select_rs<float>, G, max_gv, 4, c_out[1], dyn_out[1]);
    grid_out[0] = grid_cost(dtype, false, G, max_ge) < t_rbp ? 1 : 0;
    grid_out[1] = grid_cost(dtype, true, G, max_gv) < t_rs ? 1 : 0;
}

template <typename K>
static void launch_clustered(K kernel, int which, const DevGraph &g, const DevRun &dr, const RunParams &rp,
                             cudaStream_t s)
{
    const unsigned C = (unsigned)std::max(1, g.sel_c[which]);
    DevGraph gl = g;
    gl.sel_smem_bytes = g.sel_dyn[which];   // the kernels stage a slice only when it fits this size
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.G * C, 1, 1);
    cfg.blockDim = dim3(SEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)gl.sel_smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, gl, dr, rp);
}

void launch_select_rbp(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    if (g.sel_grid[0] && dr.gsel) {
        launch_select_rbp_grid(dtype, g, dr, rp, s);
        return;
    }
    switch (dtype) {
    case DT_F64: launch_clustered(k_select_rbp<double>, 0, g, dr, rp, s); break;
    case DT_F32: launch_clustered(k_select_rbp<float>, 0, g, dr, rp, s); break;
    case DT_BF16: launch_clustered(k_select_rbp<__nv_bfloat16>, 0, g, dr, rp, s); break;
    default: launch_clustered(k_select_rbp<int16_t>, 0, g, dr, rp, s); break;
    }
}

void launch_select_rs(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    if (g.sel_grid[1] && dr.gsel) {
        launch_select_rs_grid(dtype, g, dr, rp, s);
        return;
    }
    // selection reads residuals only: FP64 runs keep double residuals, the others float
    if (dtype == DT_F64)
        launch_clustered(k_select_rs<double>, 1, g, dr, rp, s);
    else
        launch_clustered(k_select_rs<float>, 1, g, dr, rp, s);
}

}  // namespace bpg
