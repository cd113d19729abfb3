// Persistent batch kernel: every round of Algorithm 1 for a batch of binary
// Ising graphs in one launch.
//
// A thread-block cluster of C CTAs owns one graph at a time and runs all of its
// rounds; graphs are claimed from a device work counter, so a grid of
// (SMs / C) clusters works through thousands of graphs of uneven sizes. Each
// CTA owns a contiguous slice of the graph's vertices (and so of its CSR
// edges). The phases of a round are separated by cluster barriers (hardware
// barrier.cluster, no spin-waits):
//   eval      every out-message of the slice's vertices (eval_vertex_bin), the
//             CTA's max residual / unconverged count in shared memory
//   decide    every CTA sums the cluster's partials through distributed shared
//             memory and takes the same decision (eps test, max rounds, budget,
//             RnBP EdgeRatio p, RBP/RS frontier size)
//   frontier  LBP: buffer swap; RnBP: eps filter + Philox on the slice's edges;
//             RBP: cluster top-k + commit; RS: vertex residual, cluster top-k
//             roots, BFS levels, splash sweep (commit fused with next level)
// There is no dependence between clusters. The arithmetic is the per-round
// kernels' (shared device functions), so results are bit-identical.
#include "bp_internal.cuh"
#include "bp_launch.h"
#include "bp_select.cuh"
#include "bp_update.cuh"

namespace bpg {

constexpr int PT_THREADS = 1024;
static_assert(PT_THREADS == SEL_THREADS, "the cluster select scans assume SEL_THREADS threads per CTA");

struct PtShared {
    double part_max;                 // this CTA's largest residual of the evaluation
    unsigned long long part_cnt;     // this CTA's messages with residual >= eps
    int graph;                       // rank 0: graph claimed for the cluster
    int stop;                        // rank 0: wall-clock budget exhausted
    double w_max[32];
    unsigned long long w_cnt[32];
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Block-wide (max, sum); the result is valid in thread 0.
__device__ __forceinline__ void block_max_sum(PtShared &ps, double m, unsigned long long c, double &om,
                                              unsigned long long &oc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        ps.w_max[warp] = m;
        ps.w_cnt[warp] = c;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        m = lane < nw ? ps.w_max[lane] : 0.0;
        c = lane < nw ? ps.w_cnt[lane] : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
    }
    om = m;
    oc = c;
    __syncthreads();
}

template <typename S, int SCHED>
__global__ void __launch_bounds__(PT_THREADS) k_persistent(DevGraph g, DevRun dr, RunParams rp, long long budget_ns)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    using KeyT = decltype(key_bits((RT)0));
    __shared__ SelShared<KeyT> sh;
    __shared__ PtShared ps;
    extern __shared__ __align__(16) unsigned char pt_smem[];
    cg::cluster_group cl = cg::this_cluster();
    const unsigned C = cl.num_blocks(), rank = cl.block_rank();
    const A eps_a = eps_in(rp, (A)0);
    RT *R = (RT *)dr.resid;
    const unsigned long long t0 = global_ns();

    for (;;) {
        if (rank == 0 && threadIdx.x == 0)
            ps.graph = atomicAdd(dr.queue, 1);
        cl.sync();
        const int gg = *cl.map_shared_rank(&ps.graph, 0);
        cl.sync();   // every CTA has read the claim before any CTA may leave
        if (gg >= g.G)
            break;
        const int v0 = g.gv_off[gg], nv = g.gv_off[gg + 1] - v0;
        const int ge0 = g.ge_off[gg], Mg = g.ge_off[gg + 1] - ge0;
        int vlo, vhi;
        slice_of(nv, rank, C, vlo, vhi);
        const int elo = g.row_ptr[v0 + vlo] - ge0, ehi = g.row_ptr[v0 + vhi] - ge0;
        int rounds = 0, cur = 0, status = ST_RUNNING, evaluations = 0;
        unsigned long long n_prev = 0, rbp_committed = 0;
        unsigned long long my_commit = 0, my_splash = 0;   // this thread's
        double final_maxr = 0.0;
        unsigned long long final_cnt = 0;

        for (;;) {
            // ---- full evaluation of the slice's vertices (Eq. 2, Eq. 4)
            A maxa = 0;
            unsigned int cnt = 0;
            {
                const S *curb = (const S *)msg_buf(dr, cur);
                S *outb = (S *)msg_buf(dr, cur ^ 1);
                for (int t = vlo + (int)threadIdx.x; t < vhi; t += blockDim.x)
                    eval_vertex_bin<S, SCHED != SCHED_LBP>(g, curb, outb, R, v0 + t, eps_a, maxa, cnt);
            }
            double bm;
            unsigned long long bc;
            block_max_sum(ps, (double)maxa, (unsigned long long)cnt, bm, bc);
            if (threadIdx.x == 0) {
                ps.part_max = bm;
                ps.part_cnt = bc;
                if (rank == 0)
                    ps.stop = (budget_ns > 0 && (long long)(global_ns() - t0) > budget_ns) ? 1 : 0;
            }
            cl.sync();
            // ---- decide (every thread of every CTA computes the same)
            double maxr = 0.0;
            unsigned long long ntot = 0;
            for (unsigned r = 0; r < C; ++r) {
                const PtShared *p = cl.map_shared_rank(&ps, r);
                maxr = fmax(maxr, p->part_max);
                ntot += p->part_cnt;
            }
            const int stop = cl.map_shared_rank(&ps, 0)->stop;
            cl.sync();   // partials are read by everyone before they change
            ++evaluations;
            final_maxr = maxr;
            final_cnt = ntot;
            if (maxr < rp.eps) {
                status = ST_CONVERGED;
                break;
            }
            if (rounds >= rp.max_rounds) {
                status = ST_MAXROUNDS;
                break;
            }
            if (stop) {
                status = ST_STOPPED;
                break;
            }
            ++rounds;
            const bool tr = rp.record_trace && rounds <= rp.trace_capacity;
            // ---- frontier
            if (SCHED == SCHED_LBP) {
                cur ^= 1;
            } else if (SCHED == SCHED_RNBP) {
                const double p = edge_ratio_p(rp, graph_low_p(dr, rp, gg), rounds, ntot, n_prev);
                GState sel;
                rnbp_threshold(p, sel.thr, sel.always);
                S *dst = (S *)dr.msg[0];
                const S *src = (const S *)dr.msg[1];
                for (int e = elo + (int)threadIdx.x; e < ehi; e += blockDim.x) {
                    const int ge = ge0 + e;
                    if (R[ge] >= eps_in(rp, (RT)0) &&
                        rnbp_pick(rp, (uint32_t)e, (uint32_t)rounds, (uint32_t)gg, sel)) {
                        dst[ge] = src[ge];
                        ++my_commit;
                        if (tr)
                            atomicOr(&dr.trace[(size_t)(rounds - 1) * rp.trace_words + (ge >> 5)], 1u << (ge & 31));
                    }
                }
            } else if (SCHED == SCHED_RBP) {
                const double p = rp.dynamic_p ? edge_ratio_p(rp, graph_low_p(dr, rp, gg), rounds, ntot, n_prev)
                                              : graph_low_p(dr, rp, gg);
                double v = ceil(p * (double)Mg);
                long long kk = (v > (double)Mg) ? Mg : (long long)v;
                kk = kk < 1 ? 1 : (kk > Mg ? Mg : kk);
                rbp_committed += (unsigned long long)kk;
                const int nl = ehi - elo;
                const RT *Rs = R + ge0 + elo;
                KeyT *s_keys = reinterpret_cast<KeyT *>(pt_smem);
                const bool staged = (size_t)nl * sizeof(KeyT) <= (size_t)g.sel_smem_bytes;
                if (staged)
                    stage_keys<KeyT>(nl, s_keys, [&](int idx) { return key_bits(Rs[idx]); });
                auto key = [&](int idx) -> KeyT { return staged ? s_keys[idx] : key_bits(Rs[idx]); };
                KeyT thr;
                int take_eq, eq_total;
                cluster_select_threshold<KeyT>(cl, sh, nl, (int)kk, key, thr, take_eq, eq_total);
                S *dst = (S *)dr.msg[0];
                const S *src = (const S *)dr.msg[1];
                cluster_select_apply<KeyT>(cl, sh, nl, thr, take_eq, eq_total, key, [&](int idx, bool take) {
                    if (!take)
                        return;
                    const int ge = ge0 + elo + idx;
                    dst[ge] = src[ge];
                    if (tr)
                        atomicOr(&dr.trace[(size_t)(rounds - 1) * rp.trace_words + (ge >> 5)], 1u << (ge & 31));
                });
            } else {   // SCHED_RS
                const int64_t base = (rp.rs_roots_mode == 1) ? nv : Mg;
                const double p = rp.dynamic_p ? edge_ratio_p(rp, graph_low_p(dr, rp, gg), rounds, ntot, n_prev)
                                              : graph_low_p(dr, rp, gg);
                double v = ceil(p * (double)base);
                long long kk = (v > (double)nv) ? nv : (long long)v;
                kk = kk < 1 ? 1 : (kk > nv ? nv : kk);
                const int nl = vhi - vlo;
                const bool staged = (size_t)nl * sizeof(KeyT) <= (size_t)g.sel_smem_bytes;
                KeyT *vkeys = staged ? reinterpret_cast<KeyT *>(pt_smem)
                                     : reinterpret_cast<KeyT *>(dr.vres) + v0 + vlo;
                // vertex residual: max residual of the messages into the vertex
                for (int idx = threadIdx.x; idx < nl; idx += blockDim.x) {
                    const int vv = v0 + vlo + idx;
                    RT m = 0;
                    for (int f = g.row_ptr[vv]; f < g.row_ptr[vv + 1]; ++f) {
                        const RT r = R[g.rev[f]];
                        m = r > m ? r : m;
                    }
                    vkeys[idx] = key_bits(m);
                }
                __syncthreads();
                auto key = [&](int idx) -> KeyT { return vkeys[idx]; };
                KeyT thr;
                int take_eq, eq_total;
                cluster_select_threshold<KeyT>(cl, sh, nl, (int)kk, key, thr, take_eq, eq_total);
                cluster_select_apply<KeyT>(cl, sh, nl, thr, take_eq, eq_total, key, [&](int idx, bool take) {
                    const int vv = v0 + vlo + idx;
                    dr.level[vv] = take ? (int8_t)0 : (int8_t)-1;
                    if (take && tr)
                        atomicOr(&dr.trace[(size_t)(rounds - 1) * rp.trace_words + (vv >> 5)], 1u << (vv & 31));
                });
                cl.sync();
                const int h = rp.splash_depth;
                for (int d = 1; d <= h; ++d) {
                    for (int t = vlo + (int)threadIdx.x; t < vhi; t += blockDim.x)
                        bfs_vertex(g, dr, v0 + t, d);
                    cl.sync();
                }
                auto level_of = [h](int step) { return step <= h ? h - step : step - h; };
                for (int step = -1; step <= 2 * h; ++step) {
                    const int Lc = step >= 0 ? level_of(step) : -1;
                    const int Le = step < 2 * h ? level_of(step + 1) : -1;
                    for (int t = vlo + (int)threadIdx.x; t < vhi; t += blockDim.x) {
                        const int vv = v0 + t;
                        const unsigned c = splash_vertex_bin<S>(g, dr, vv, dr.level[vv], Lc, Le);
                        my_commit += c;
                        my_splash += c;
                    }
                    cl.sync();
                }
            }
            n_prev = ntot;
            cl.sync();   // frontier writes are visible before the next evaluation
        }

        // ---- results of graph gg
        double unused;
        unsigned long long cta_commit, cta_splash;
        block_max_sum(ps, 0.0, my_commit, unused, cta_commit);
        block_max_sum(ps, 0.0, my_splash, unused, cta_splash);
        if (threadIdx.x == 0) {
            GState *st = dr.gs + gg;
            if (cta_commit)
                atomicAdd(&st->committed, cta_commit);
            if (cta_splash)
                atomicAdd(&st->evals, cta_splash);
            if (rank == 0) {
                const unsigned long long full = (unsigned long long)evaluations * (unsigned long long)Mg;
                atomicAdd(&st->evals, full);
                if (SCHED == SCHED_LBP)
                    atomicAdd(&st->committed, (unsigned long long)rounds * (unsigned long long)Mg);
                if (SCHED == SCHED_RBP)
                    atomicAdd(&st->committed, rbp_committed);
                st->full_evals = full;
                st->full_nodes = (unsigned long long)evaluations * (unsigned long long)nv;
                st->status = status;
                st->rounds = rounds;
                st->cur = cur;
                st->final_maxr = final_maxr;
                st->final_cnt = final_cnt;
                st->n_prev = n_prev;
                atomicSub(dr.n_running, 1);
            }
        }
        cl.sync();   // ps.graph is rewritten only after every CTA has left this graph
    }
}

static unsigned persistent_cluster_size(const DevGraph &g, int max_slice_keys_bytes_needed)
{
    (void)max_slice_keys_bytes_needed;
    int c = 152 / (g.G > 0 ? g.G : 1);
    c = c < 1 ? 1 : (c > 8 ? 8 : c);
    return (unsigned)c;
}

template <typename S, int SCHED> static cudaError_t launch_pt(const DevGraph &g, const DevRun &dr,
                                                               const RunParams &rp, long long budget_ns,
                                                               cudaStream_t s)
{
    auto kernel = k_persistent<S, SCHED>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SEL_SMEM_BYTES);
        attr_set = true;
    }
    const unsigned C = persistent_cluster_size(g, 0);
    unsigned clusters = 152 / C;
    if (clusters > (unsigned)g.G)
        clusters = (unsigned)g.G;
    if (clusters < 1)
        clusters = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * C, 1, 1);
    cfg.blockDim = dim3(PT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)g.sel_smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, g, dr, rp, budget_ns);
}

template <typename S>
static cudaError_t launch_pt_sched(const DevGraph &g, const DevRun &dr, const RunParams &rp, long long budget_ns,
                                   cudaStream_t s)
{
    switch (rp.schedule) {
    case SCHED_LBP: return launch_pt<S, SCHED_LBP>(g, dr, rp, budget_ns, s);
    case SCHED_RNBP: return launch_pt<S, SCHED_RNBP>(g, dr, rp, budget_ns, s);
    case SCHED_RBP: return launch_pt<S, SCHED_RBP>(g, dr, rp, budget_ns, s);
    default: return launch_pt<S, SCHED_RS>(g, dr, rp, budget_ns, s);
    }
}

cudaError_t launch_persistent(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp,
                              long long budget_ns, cudaStream_t s)
{
    switch (dtype) {
    case DT_F64: return launch_pt_sched<double>(g, dr, rp, budget_ns, s);
    case DT_F32: return launch_pt_sched<float>(g, dr, rp, budget_ns, s);
    case DT_BF16: return launch_pt_sched<__nv_bfloat16>(g, dr, rp, budget_ns, s);
    default: return launch_pt_sched<int16_t>(g, dr, rp, budget_ns, s);
    }
}

}  // namespace bpg
