// Round kernels of frontier-scheduled loopy BP on sm_103a.
//
// One round of Algorithm 1 on the device:
//   eval    candidates of Eq. 2 for every message of every running graph, the
//           residual of Eq. 4 (max-norm of the probability-domain change) fused
//           in the epilogue, and the per-graph max-residual / unconverged count
//   decide  per graph: eps test, max-rounds test, the next frontier's size or
//           RnBP probability (EdgeRatio, Section IV-A)
//   commit  LBP: swap buffers; RnBP: eps filter + Philox Bernoulli; RBP/RS: in
//           the select kernels (bp_select.cu)
// Messages live in the log domain: binary messages as one log-odds value
// u = log m(1) - log m(0), k-state messages as k normalised logs.
#include "bp_internal.cuh"
#include "bp_launch.h"
#include "bp_update.cuh"

#include <math.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

namespace bpg {

constexpr int BLOCK = 256;

// --------------------------------------------------------------------------
// Binary Ising messages, one thread per vertex: the thread gathers the
// incoming log-odds of its vertex through rev[], forms the cavity of each
// out-edge by subtraction and writes every out-message of the vertex
// (eval_vertex_bin). Full evaluations only (LBP and the frontier modes).
template <typename S, int MODE>
__global__ void __launch_bounds__(BLOCK) k_eval_bin(DevGraph g, DevRun dr, RunParams rp)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    const int first = blockIdx.x * blockDim.x;
    const int last = min(g.n - 1, first + (int)blockDim.x - 1);
    const int g0 = g.gid[first];
    const bool uniform = (g0 == g.gid[last]);
    const int i = first + threadIdx.x;
    bool valid = false;
    int gg = g0;
    A maxa = 0;
    unsigned int cnt = 0;
    if (i < g.n) {
        gg = g.gid[i];
        if (dr.gs[gg].status == ST_RUNNING) {
            valid = true;
            const int c = dr.gs[gg].cur;
            eval_vertex_bin<S, MODE == MODE_CAND>(g, (const S *)msg_buf(dr, c), (S *)msg_buf(dr, c ^ 1),
                                                  (RT *)dr.resid, i, eps_in(rp, (A)0), maxa, cnt);
        }
    }
    reduce_to_graph(dr, uniform, g0, valid, gg, (double)maxa, cnt);
}

// The same mapping with the prefetching vertex routine (eval_vertex_bin_pf):
// graph arrays and the graph's status load in parallel. MINB = resident
// blocks per SM the register budget is fitted to.
template <typename S, int MODE, int CACHE, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_eval_bin_pf(DevGraph g, DevRun dr, RunParams rp)
{
    griddep_launch_dependents();
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    const int first = blockIdx.x * blockDim.x;
    const int last = min(g.n - 1, first + (int)blockDim.x - 1);
    const int g0 = g.gid[first];
    const bool uniform = (g0 == g.gid[last]);
    const int i = first + threadIdx.x;
    bool valid = false;
    int gg = g0;
    A maxa = 0;
    unsigned int cnt = 0;
    if (i < g.n) {
        gg = g.gid[i];
        valid = eval_vertex_bin_pf<S, MODE == MODE_CAND, CACHE, true>(g, dr, (RT *)dr.resid, i, gg,
                                                                       eps_in(rp, (A)0), maxa, cnt);
    } else {
        griddep_wait();
    }
    reduce_to_graph(dr, uniform, g0, valid, gg, (double)maxa, cnt);
}

// --------------------------------------------------------------------------
// k-state messages (k <= KP <= 32): a group of KP lanes per vertex, lane x
// holds state x. S_i(x) = theta_i(x) + sum_in l(x); per out-edge the cavity is
// S_i - l_{j->i}; with a(x) = exp(cav(x) - max cav) the new message is
// c(y) = sum_x a(x) psi(x, y), normalised, stored as log c(y).
// Lane mask of the KP-lane group that contains this thread. Groups of one warp
// may run different trip counts (vertex degrees differ), so every shuffle names
// only its own group's lanes.
template <int KP> __device__ __forceinline__ unsigned grp_mask()
{
    if (KP == 32)
        return 0xffffffffu;
    return ((1u << KP) - 1u) << ((threadIdx.x & 31) & ~(KP - 1));
}
template <int KP> __device__ __forceinline__ float grp_max(unsigned m, float v)
{
#pragma unroll
    for (int o = KP / 2; o; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(m, v, o, KP));
    return v;
}
template <int KP> __device__ __forceinline__ double grp_max(unsigned m, double v)
{
#pragma unroll
    for (int o = KP / 2; o; o >>= 1)
        v = fmax(v, __shfl_xor_sync(m, v, o, KP));
    return v;
}
template <int KP, typename T> __device__ __forceinline__ T grp_sum(unsigned m, T v)
{
#pragma unroll
    for (int o = KP / 2; o; o >>= 1)
        v += __shfl_xor_sync(m, v, o, KP);
    return v;
}

template <typename A> __device__ __forceinline__ A log_floor();
template <> __device__ __forceinline__ float log_floor<float>() { return -80.0f; }
template <> __device__ __forceinline__ double log_floor<double>() { return -700.0; }

template <typename S, int KP, int MODE>
__global__ void __launch_bounds__(BLOCK) k_eval_gen(DevGraph g, DevRun dr, RunParams rp, int level_L)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    __shared__ float s_psi[32 * 32];
    const int k = g.k;
    if (g.pair_kind == 2) {
        for (int t = threadIdx.x; t < k * k; t += blockDim.x)
            s_psi[t] = g.psi_shared[t];
        __syncthreads();
    }
    constexpr int NPB = BLOCK / KP;
    const int lane = threadIdx.x % KP;
    const int first = blockIdx.x * NPB;
    const int last = min(g.n - 1, first + NPB - 1);
    const int g0 = g.gid[first];
    const bool uniform = (g0 == g.gid[last]);
    const int i = first + (int)threadIdx.x / KP;
    const bool lane_ok = lane < k;
    bool valid = false;
    int gg = g0;
    A maxa = 0;
    const A eps_a = eps_in(rp, (A)0);
    unsigned int cnt = 0;
    bool act = false;
    if (i < g.n) {
        gg = g.gid[i];
        act = dr.gs[gg].status == ST_RUNNING;
        if (MODE == MODE_SPLASH)
            act = act && (dr.level[i] == level_L);
    }
    if (act) {   // uniform across the KP-lane group
        const unsigned gm = grp_mask<KP>();
        valid = (lane == 0);
        const int cur_idx = dr.gs[gg].cur;
        const S *cur = (const S *)msg_buf(dr, cur_idx);
        S *out = (S *)msg_buf(dr, cur_idx ^ 1);
        const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
        A Sx = lane_ok ? (A)g.unary[(size_t)i * k + lane] : (A)0;
        for (int e = beg; e < end; ++e)
            if (lane_ok)
                Sx += Store<S>::ld(cur + (size_t)g.rev[e] * k + lane, g.qscale);
        RT *R = (RT *)dr.resid;
        for (int e = beg; e < end; ++e) {
            A lin = lane_ok ? Store<S>::ld(cur + (size_t)g.rev[e] * k + lane, g.qscale) : (A)0;
            A cav = lane_ok ? Sx - lin : (A)(-1e30);
            A mx = grp_max<KP>(gm, cav);
            A a = lane_ok ? m_exp(cav - mx) : (A)0;
            A acc = 0;
            if (g.pair_kind == 2) {
                for (int x = 0; x < k; ++x) {
                    A ax = __shfl_sync(gm, a, x, KP);
                    if (lane_ok)
                        acc += ax * (A)s_psi[x * k + lane];
                }
            } else {
                const float *tab = g.pair + (size_t)e * k * k;
                for (int x = 0; x < k; ++x) {
                    A ax = __shfl_sync(gm, a, x, KP);
                    if (lane_ok)
                        acc += ax * m_exp((A)tab[x * k + lane]);
                }
            }
            A z = grp_sum<KP>(gm, lane_ok ? acc : (A)0);
            A lnew = lane_ok ? m_log(m_div(acc, z)) : (A)0;
            lnew = lnew > log_floor<A>() ? lnew : log_floor<A>();
            if (MODE == MODE_SPLASH) {
                if (lane_ok)
                    Store<S>::st(out + (size_t)e * k + lane, lnew, g.qscale);
                continue;
            }
            A pn = lane_ok ? m_exp(Store<S>::quant(lnew, g.qscale)) : (A)0;
            A po = lane_ok ? m_exp(Store<S>::ld(cur + (size_t)e * k + lane, g.qscale)) : (A)0;
            A r = grp_max<KP>(gm, fabs(pn - po));
            if (lane_ok)
                Store<S>::st(out + (size_t)e * k + lane, lnew, g.qscale);
            if (MODE == MODE_CAND && lane == 0)
                R[e] = (RT)r;
            maxa = r > maxa ? r : maxa;
            cnt += (r >= eps_a) ? 1u : 0u;
        }
    }
    if (MODE != MODE_SPLASH)
        reduce_to_graph(dr, uniform, g0, valid, gg, (double)maxa, cnt);
}

// --------------------------------------------------------------------------
// Per-graph decision after an evaluation: one warp per graph, eight graphs
// per block (a batch of thousands of graphs launches a few hundred blocks, not
// one tiny block per graph). The graph's state, its reduction sub-slots and
// its frontier fraction are independent loads, issued together; the slots of
// a stopped graph are already zero (its evaluations are skipped), so only a
// running graph clears them.
constexpr int DECIDE_BLOCK = 256;

__global__ void __launch_bounds__(DECIDE_BLOCK) k_decide(DevGraph g, DevRun dr, RunParams rp)
{
    griddep_launch_dependents();
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const int gg = (int)(((unsigned)blockIdx.x * DECIDE_BLOCK + threadIdx.x) >> 5);
    if (gg == 0 && lane <= LVL_MAX && dr.lvl_cnt)
        dr.lvl_cnt[lane] = 0;   // Residual Splash level lists of this round start empty
    if (gg >= g.G)
        return;
    GState *stp = dr.gs + gg;
    GState st = {};
    if (lane == 0)
        st = *stp;
    unsigned long long mb = dr.red_max[(size_t)gg * NSUB + lane];
    unsigned int c = dr.red_cnt[(size_t)gg * NSUB + lane];
    unsigned int cm = dr.red_commit ? dr.red_commit[(size_t)gg * NSUB + lane] : 0u;
    unsigned int cm_lo = rp.fused_rnbp ? dr.red_commit_lo[(size_t)gg * NSUB + lane] : 0u;
    const double low_p = lane == 0 ? graph_low_p(dr, rp, gg) : 0.0;
    if (__shfl_sync(0xffffffffu, st.status, 0) != ST_RUNNING)
        return;
    dr.red_max[(size_t)gg * NSUB + lane] = 0ull;
    dr.red_cnt[(size_t)gg * NSUB + lane] = 0u;
    if (dr.red_commit)
        dr.red_commit[(size_t)gg * NSUB + lane] = 0u;
    if (rp.fused_rnbp)
        dr.red_commit_lo[(size_t)gg * NSUB + lane] = 0u;
    mb = warp_max_u64(mb);
    c = warp_sum_u32(c);
    cm = warp_sum_u32(cm);
    cm_lo = warp_sum_u32(cm_lo);
    if (lane != 0)
        return;
    if (!rp.fused_rnbp)
        st.committed += (unsigned long long)cm;   // the RnBP commit of the previous round
    const double maxr = __longlong_as_double((long long)mb);
    const int64_t Mg = g.ge_off[gg + 1] - g.ge_off[gg];
    const int64_t ng = g.gv_off[gg + 1] - g.gv_off[gg];
    st.evals += (unsigned long long)Mg;
    st.full_evals += (unsigned long long)Mg;
    st.full_nodes += (unsigned long long)ng;
    st.final_maxr = maxr;
    st.final_cnt = c;
    if (maxr < rp.eps) {
        st.status = ST_CONVERGED;
    } else if (st.rounds >= rp.max_rounds) {
        st.status = ST_MAXROUNDS;
    } else {
        st.rounds += 1;
        if (rp.schedule == SCHED_LBP) {
            st.cur ^= 1;
            st.committed += (unsigned long long)Mg;
        } else if (rp.schedule == SCHED_RNBP) {
            const bool lowsel = edge_ratio_low(rp, st.rounds, c, st.n_prev);
            rnbp_threshold(lowsel ? low_p : rp.high_p, st.thr, st.always);
            if (rp.fused_rnbp) {
                // the update already wrote both outcomes: HighP into buffer
                // cur + 1, LowP into cur + 2 (mod 3)
                st.cur = (st.cur + (lowsel ? 2 : 1)) % 3;
                st.committed += (unsigned long long)(lowsel ? cm_lo : cm);
            }
        } else {
            const int64_t base = (rp.schedule == SCHED_RS && rp.rs_roots_mode == 1) ? ng : Mg;
            const int64_t hi = (rp.schedule == SCHED_RS) ? ng : Mg;
            const double p = rp.dynamic_p ? edge_ratio_p(rp, low_p, st.rounds, c, st.n_prev) : low_p;
            double v = ceil(p * (double)base);
            int64_t kk = (v > (double)hi) ? hi : (int64_t)v;
            kk = kk < 1 ? 1 : kk;
            kk = kk > hi ? hi : kk;
            st.k_sel = (int32_t)kk;
            if (rp.schedule == SCHED_RBP)
                st.committed += (unsigned long long)kk;
        }
        st.n_prev = c;
    }
    *stp = st;
    if (st.status != ST_RUNNING)
        atomicSub(dr.n_running, 1);
}

// --------------------------------------------------------------------------
// Per-vertex block reduction of a count into gs[g].committed (and evals).
__device__ __forceinline__ void add_commit_counts(const DevRun &dr, bool uniform, int g0, bool valid,
                                                  int g, unsigned int c, bool also_evals)
{
    if (uniform) {
        __shared__ unsigned int s_c[32];
        unsigned int v = warp_sum_u32(valid ? c : 0u);
        int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0)
            s_c[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int nw = (blockDim.x + 31) >> 5;
            v = lane < nw ? s_c[lane] : 0u;
            v = warp_sum_u32(v);
            if (lane == 0 && v) {
                atomicAdd(&dr.gs[g0].committed, (unsigned long long)v);
                if (also_evals)
                    atomicAdd(&dr.gs[g0].evals, (unsigned long long)v);
            }
        }
    } else if (valid && c) {
        atomicAdd(&dr.gs[g].committed, (unsigned long long)c);
        if (also_evals)
            atomicAdd(&dr.gs[g].evals, (unsigned long long)c);
    }
}

// --------------------------------------------------------------------------
// Vertex tiles of the fallback RnBP commit (k_commit_rnbp_tiled): 256
// consecutive vertices and their contiguous edge range, up to TILE_E edges
// staged per tile.
constexpr int TILE_V = 256;
constexpr int TILE_E = 8 * TILE_V - 8;

// Lanes per tile of the warp-tile RnBP commits. A tile of <= 128 messages
// meets <= 17 aligned octets of its graph (the messages of one Philox block),
// so a lane takes COMMIT_OPL = 3 octets: its eligibility and pick bits fit
// one word.
constexpr int COMMIT_LPT = 8;
constexpr int COMMIT_OPL = (STREAM_WT / RNBP_PER_BLOCK + 1 + COMMIT_LPT - 1) / COMMIT_LPT;
static_assert(COMMIT_OPL * RNBP_PER_BLOCK <= 32, "a lane's eligibility and pick bits fit one word");

// Picks of a lane's octets: bit (8 k + j) of elig is message j of the lane's
// octet k (octet oct0 + hl + COMMIT_LPT k of graph gg); the octet's Philox
// block is drawn only when one of its messages is eligible.
__device__ __forceinline__ unsigned commit_picks(const RunParams &rp, unsigned elig, int oct0, int hl, int rounds,
                                                 int gg, bool always, uint32_t thr)
{
    unsigned pick = 0;
#pragma unroll
    for (int k = 0; k < COMMIT_OPL; ++k) {
        const unsigned b8 = (elig >> (RNBP_PER_BLOCK * k)) & 0xffu;
        if (!b8)
            continue;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (!always)
            w = rnbp_block(rp, (uint32_t)(oct0 + hl + COMMIT_LPT * k), (uint32_t)rounds, (uint32_t)gg);
#pragma unroll
        for (int j = 0; j < RNBP_PER_BLOCK; ++j)
            if (((b8 >> j) & 1u) && (always || rnbp_draw16(w, (uint32_t)j) < thr))
                pick |= 1u << (RNBP_PER_BLOCK * k + j);
    }
    return pick;
}

// Copies a lane's picked candidates (bit b: message first + 8 (hl +
// COMMIT_LPT (b / 8)) + b % 8, epm stored elements each) into the committed
// buffer, for binary messages every load before any store, and records them
// in the round's trace.
template <typename S>
__device__ __forceinline__ void commit_copy(const DevRun &dr, const RunParams &rp, unsigned pick, int first, int hl,
                                            int rounds, int epm)
{
    S *dst = (S *)dr.msg[0];
    const S *src = (const S *)dr.msg[1];
    constexpr int NB = COMMIT_OPL * RNBP_PER_BLOCK;
    if (epm == 1) {
        S v[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (pick >> b & 1u)
                v[b] = src[first + RNBP_PER_BLOCK * (hl + COMMIT_LPT * (b / RNBP_PER_BLOCK)) + b % RNBP_PER_BLOCK];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (pick >> b & 1u)
                dst[first + RNBP_PER_BLOCK * (hl + COMMIT_LPT * (b / RNBP_PER_BLOCK)) + b % RNBP_PER_BLOCK] = v[b];
    } else {
        for (int b = 0; b < NB; ++b)
            if (pick >> b & 1u) {
                const size_t e =
                    (size_t)(first + RNBP_PER_BLOCK * (hl + COMMIT_LPT * (b / RNBP_PER_BLOCK)) + b % RNBP_PER_BLOCK);
                for (int x = 0; x < epm; ++x)
                    dst[e * epm + x] = src[e * epm + x];
            }
    }
    if (rp.record_trace && rounds <= rp.trace_capacity) {
        for (int b = 0; b < NB; ++b)
            if (pick >> b & 1u) {
                const int e = first + RNBP_PER_BLOCK * (hl + COMMIT_LPT * (b / RNBP_PER_BLOCK)) + b % RNBP_PER_BLOCK;
                atomicOr(&dr.trace[(size_t)(rounds - 1) * rp.trace_words + (e >> 5)], 1u << (e & 31));
            }
    }
}

// RnBP commit over the warp tiles of the streamed update (single-graph runs
// of consecutive vertices, <= 128 out-edges), from the residuals (the other
// update mappings and k-state messages): eight lanes per tile (a warp
// carries four tiles' loads in flight) read the tile's commit record, then
// together the graph's round state and the eps test of the tile's messages.
// Each lane takes aligned octets of consecutive messages of the graph, which
// share one Philox block, applies the eps filter and the random filter, then
// issues the loads of all its selected candidates before any store. The
// commits of a tile are added with one atomic.
template <typename S>
__global__ void __launch_bounds__(BLOCK, 5) k_commit_rnbp_wt(DevGraph g, DevRun dr, RunParams rp)
{
    griddep_launch_dependents();
    using RT = typename ResidT<S>::T;
    constexpr int LPT = COMMIT_LPT;
    const int lane = threadIdx.x & 31, hl = lane % LPT;
    const unsigned hmask = ((1u << LPT) - 1u) << (lane - hl);
    const int t = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) / LPT);   // this lane group's tile
    const int4 rc = t < g.n_wtiles ? g.ctiles[t] : make_int4(0, 0, 0, 0);   // {e0, e1, graph, graph's e0}
    const int e0 = rc.x, e1 = rc.y, gg = rc.z, ge0 = rc.w;
    const int off = (e0 - ge0) & (RNBP_PER_BLOCK - 1);   // the first octet starts up to 7 messages before the tile
    griddep_wait();   // residuals, candidates and round state come from the previous kernels
    if (e1 <= e0)
        return;   // the whole lane group: a tile past the end or without edges
    const GState *sp = dr.gs + gg;
    const int status = sp->status, rounds = sp->rounds, always = sp->always;
    const uint32_t thr = sp->thr;
    // eligibility: residual >= eps (Eq. 4 against eps)
    unsigned elig = 0;
    if (status == ST_RUNNING) {
        const RT *R = (const RT *)dr.resid;
        const RT eps = eps_in(rp, (RT)0);
#pragma unroll
        for (int b = 0; b < COMMIT_OPL * RNBP_PER_BLOCK; ++b) {
            const int e = e0 - off + RNBP_PER_BLOCK * (hl + LPT * (b / RNBP_PER_BLOCK)) + b % RNBP_PER_BLOCK;
            if (e >= e0 && e < e1 && R[e] >= eps)
                elig |= 1u << b;
        }
    }
    const unsigned pick = commit_picks(rp, elig, (e0 - ge0 - off) / RNBP_PER_BLOCK, hl, rounds, gg, always != 0, thr);
    commit_copy<S>(dr, rp, pick, e0 - off, hl, rounds, g.epm);
    // one atomic per tile into one of the graph's sub-slots (a single-graph
    // run has tens of thousands of tiles: one counter would serialise them)
    const unsigned c = __reduce_add_sync(hmask, (unsigned)__popc(pick));
    if (hl == 0 && c)
        atomicAdd(&dr.red_commit[(size_t)gg * NSUB + (t & (NSUB - 1))], c);
}

// RnBP commit after the streamed update (binary messages), from the four
// flag words per warp tile that the update wrote with warp ballots (bit i:
// message i of the tile passed the eps test of Eq. 4; bits past the tile's
// messages are 0). A persistent grid of eight-lane groups walks the tiles with
// a stride of the group count and keeps three tiles in flight: it picks and
// copies the messages of one tile while the flag words and round state of
// its next tile and the commit record of the one after are on their way.
// Each lane takes aligned octets of consecutive messages of the graph (one
// Philox block per octet) and issues the loads of all its selected
// candidates before any store.
template <typename S>
__global__ void __launch_bounds__(BLOCK, 3) k_commit_rnbp_pipe(DevGraph g, DevRun dr, RunParams rp)
{
    griddep_launch_dependents();
    constexpr int LPT = COMMIT_LPT;
    const int lane = threadIdx.x & 31, hl = lane % LPT;
    const unsigned hmask = ((1u << LPT) - 1u) << (lane - hl);
    const int nt = g.n_wtiles;
    const int ng = (int)(((long long)gridDim.x * blockDim.x) / LPT);   // lane groups in the grid
    int t = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) / LPT);
    const int4 z4 = make_int4(0, 0, 0, 0);
    // commit records {e0, e1, graph, graph's e0} of this tile and the next
    int4 rc = t < nt ? g.ctiles[t] : z4;
    int4 rn = (long long)t + ng < nt ? g.ctiles[t + ng] : z4;
    griddep_wait();   // flags, candidates and round state come from the previous kernels
    // flag words and round state (status, rounds, always, thr) of tile t
    uint4 fw = make_uint4(0u, 0u, 0u, 0u);
    int4 st = z4;
    if (t < nt) {
        fw = *reinterpret_cast<const uint4 *>(dr.eps_words + (size_t)t * 4);
        const GState *sp = dr.gs + rc.z;
        st = make_int4(sp->status, sp->rounds, sp->always, (int)sp->thr);
    }
    for (; t < nt; t += ng) {
        // prefetch: the next tile's flags and state, the record after it
        const long long tn = (long long)t + ng, t2 = tn + ng;
        const int4 r2 = t2 < nt ? g.ctiles[t2] : z4;
        uint4 fwn = make_uint4(0u, 0u, 0u, 0u);
        int4 stn = z4;
        if (tn < nt) {
            fwn = *reinterpret_cast<const uint4 *>(dr.eps_words + (size_t)tn * 4);
            const GState *sp = dr.gs + rn.z;
            stn = make_int4(sp->status, sp->rounds, sp->always, (int)sp->thr);
        }
        // this tile
        const int e0 = rc.x, e1 = rc.y, gg = rc.z, ge0 = rc.w;
        const int off = (e0 - ge0) & (RNBP_PER_BLOCK - 1);   // the first octet starts up to 7 messages before the tile
        unsigned elig = 0;
        if (st.x == ST_RUNNING && e1 > e0) {
#pragma unroll
            for (int k = 0; k < COMMIT_OPL; ++k) {
                const int li0 = RNBP_PER_BLOCK * (hl + LPT * k) - off;   // the octet's first message in the tile
                unsigned b8 = 0;
                if (li0 < 0) {
                    b8 = fw.x << (-li0);
                } else if (li0 < STREAM_WT) {
                    const int wi = li0 >> 5;
                    const uint32_t lo = wi == 0 ? fw.x : (wi == 1 ? fw.y : (wi == 2 ? fw.z : fw.w));
                    const uint32_t hi = wi == 0 ? fw.y : (wi == 1 ? fw.z : (wi == 2 ? fw.w : 0u));
                    b8 = __funnelshift_r(lo, hi, li0 & 31);
                }
                elig |= (b8 & 0xffu) << (RNBP_PER_BLOCK * k);
            }
        }
        const unsigned pick = commit_picks(rp, elig, (e0 - ge0 - off) / RNBP_PER_BLOCK, hl, st.y, gg, st.z != 0,
                                           (uint32_t)st.w);
        commit_copy<S>(dr, rp, pick, e0 - off, hl, st.y, 1);
        // one atomic per tile into one of the graph's sub-slots
        const unsigned c = __reduce_add_sync(hmask, (unsigned)__popc(pick));
        if (hl == 0 && c)
            atomicAdd(&dr.red_commit[(size_t)gg * NSUB + (t & (NSUB - 1))], c);
        rc = rn;
        rn = r2;
        fw = fwn;
        st = stn;
    }
}

template <typename S> int commit_pipe_blocks()
{
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    std::call_once(once[dev], [&] {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_commit_rnbp_pipe<S>, BLOCK, 0) != cudaSuccess)
            nb = 1;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = std::max(nb, 1) * std::max(sms, 1);
    });
    return cached[dev];
}

template <typename S>
__global__ void __launch_bounds__(TILE_V) k_commit_rnbp_tiled(DevGraph g, DevRun dr, RunParams rp)
{
    griddep_launch_dependents();
    griddep_wait();
    using RT = typename ResidT<S>::T;
    __shared__ uint8_t s_src[TILE_E];
    __shared__ int s_g[TILE_V];
    const int v0 = blockIdx.x * TILE_V;
    const int nv = min(TILE_V, g.n - v0);
    const int e0 = g.row_ptr[v0];
    const int ne = g.row_ptr[v0 + nv] - e0;
    const int g0 = g.gid[v0];
    const bool uniform = (g0 == g.gid[v0 + nv - 1]);
    const int vl = threadIdx.x;
    const int v = v0 + vl;
    const RT *R = (const RT *)dr.resid;
    S *dst = (S *)dr.msg[0];
    const S *src = (const S *)dr.msg[1];
    const int epm = g.epm;
    unsigned int c = 0;
    if (ne > TILE_E) {
        bool valid = false;
        int gg = g0;
        if (vl < nv) {
            gg = g.gid[v];
            const GState st = dr.gs[gg];
            if (st.status == ST_RUNNING) {
                valid = true;
                const int ge0 = g.ge_off[gg];
                const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
                for (int e = g.row_ptr[v]; e < g.row_ptr[v + 1]; ++e) {
                    if (R[e] >= eps_in(rp, (RT)0) &&
                        rnbp_pick(rp, (uint32_t)(e - ge0), (uint32_t)st.rounds, (uint32_t)gg, st)) {
                        for (int x = 0; x < epm; ++x)
                            dst[(size_t)e * epm + x] = src[(size_t)e * epm + x];
                        ++c;
                        if (tr)
                            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (e >> 5)],
                                     1u << (e & 31));
                    }
                }
            }
        }
        add_commit_counts(dr, uniform, g0, valid, gg, c, false);
        return;
    }
    if (uniform) {
        // one graph in the tile: its round state once, every residual of the
        // tile's edges loaded up front (up to TILE_E / TILE_V per thread)
        const GState st = dr.gs[g0];
        const bool run = st.status == ST_RUNNING;
        if (run) {
            const int ge0 = g.ge_off[g0];
            const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
            constexpr int J = (TILE_E + TILE_V - 1) / TILE_V;
            RT r[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int t = vl + j * TILE_V;
                r[j] = t < ne ? R[e0 + t] : (RT)0;
            }
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int t = vl + j * TILE_V;
                const int e = e0 + t;
                if (t < ne && r[j] >= eps_in(rp, (RT)0) &&
                    rnbp_pick(rp, (uint32_t)(e - ge0), (uint32_t)st.rounds, (uint32_t)g0, st)) {
                    for (int x = 0; x < epm; ++x)
                        dst[(size_t)e * epm + x] = src[(size_t)e * epm + x];
                    ++c;
                    if (tr)
                        atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (e >> 5)], 1u << (e & 31));
                }
            }
        }
        add_commit_counts(dr, true, g0, run, g0, c, false);
        return;
    }
    if (vl < nv) {
        const int gg = g.gid[v];
        s_g[vl] = dr.gs[gg].status == ST_RUNNING ? gg : -1;
        for (int t = g.row_ptr[v] - e0; t < g.row_ptr[v + 1] - e0; ++t)
            s_src[t] = (uint8_t)vl;
    }
    __syncthreads();
    for (int t = vl; t < ne; t += TILE_V) {
        const int gg = s_g[s_src[t]];
        if (gg < 0)
            continue;
        const int e = e0 + t;
        if (R[e] < eps_in(rp, (RT)0))
            continue;
        const GState &st = dr.gs[gg];
        if (!rnbp_pick(rp, (uint32_t)(e - g.ge_off[gg]), (uint32_t)st.rounds, (uint32_t)gg, st))
            continue;
        for (int x = 0; x < epm; ++x)
            dst[(size_t)e * epm + x] = src[(size_t)e * epm + x];
        if (uniform)
            ++c;
        else
            atomicAdd(&dr.gs[gg].committed, 1ull);
        if (rp.record_trace && st.rounds <= rp.trace_capacity)
            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (e >> 5)], 1u << (e & 31));
    }
    add_commit_counts(dr, uniform, g0, uniform, g0, c, false);
}

// Residual Splash: one BFS level (pull): an unreached vertex next to a vertex of
// level d-1 gets level d.
__global__ void __launch_bounds__(BLOCK) k_bfs_level(DevGraph g, DevRun dr, int d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n)
        return;
    if (dr.gs[g.gid[i]].status != ST_RUNNING)
        return;
    bfs_vertex(g, dr, i, d);
}

// Residual Splash sub-step commit: out-messages of level-L vertices.
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_splash_commit(DevGraph g, DevRun dr, int level_L)
{
    const int first = blockIdx.x * blockDim.x;
    const int last = min(g.n - 1, first + (int)blockDim.x - 1);
    const int g0 = g.gid[first];
    const bool uniform = (g0 == g.gid[last]);
    const int i = first + threadIdx.x;
    bool valid = false;
    int gg = g0;
    unsigned int c = 0;
    if (i < g.n) {
        gg = g.gid[i];
        if (dr.gs[gg].status == ST_RUNNING && dr.level[i] == level_L) {
            valid = true;
            S *dst = (S *)dr.msg[0];
            const S *src = (const S *)dr.msg[1];
            const int epm = g.epm;
            const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
            for (int t = beg * epm; t < end * epm; ++t)
                dst[t] = src[t];
            c = (unsigned int)(end - beg);
        }
    }
    add_commit_counts(dr, uniform, g0, valid, gg, c, true);
}

// Residual Splash, binary messages: commit of one sweep level fused with the
// evaluation of the next. Vertices at level Lc copy their out-messages from
// the candidate buffer (1) to the state buffer (0); vertices at level Le
// compute new out-messages into buffer 1, reading an incoming message from
// buffer 1 when its source is at level Lc (written by the previous sub-step,
// committed by this one) and from buffer 0 otherwise. Consecutive sweep levels
// differ, so the copies and the new candidates touch disjoint messages.
// Lc = -1: evaluation only (first sub-step); Le = -1: commit only (last).
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_splash_step(DevGraph g, DevRun dr, int Lc, int Le)
{
    const int first = blockIdx.x * blockDim.x;
    const int last = min(g.n - 1, first + (int)blockDim.x - 1);
    const int g0 = g.gid[first];
    const bool uniform = (g0 == g.gid[last]);
    const int i = first + threadIdx.x;
    bool valid = false;
    int gg = g0;
    unsigned int c = 0;
    if (i < g.n) {
        gg = g.gid[i];
        if (dr.gs[gg].status == ST_RUNNING) {
            c = splash_vertex_bin<S>(g, dr, i, dr.level[i], Lc, Le);
            valid = c > 0;
        }
    }
    add_commit_counts(dr, uniform, g0, valid, gg, c, true);
}

// Residual Splash, last BFS level (pull, level d; d = 0: no BFS step, the
// splash has depth 0) fused with the per-level vertex lists of the sweeps:
// every vertex of a running graph with a level L <= h is appended to list L
// (warp-aggregated, ascending within a warp). The per-graph counts of the
// round's splash (a level-0 vertex is evaluated and committed once, a deeper
// one twice: the sweep visits levels h..1 on the way down and up) are added
// here, so the sweep kernels count nothing.
__global__ void __launch_bounds__(BLOCK) k_bfs_level_lists(DevGraph g, DevRun dr, int d, int h)
{
    const int first = blockIdx.x * blockDim.x;
    const int last = min(g.n - 1, first + (int)blockDim.x - 1);
    const int g0 = g.gid[first];
    const bool uniform = (g0 == g.gid[last]);
    const int i = first + threadIdx.x;
    int gg = g0;
    int lv = -1;
    unsigned int c = 0;
    if (i < g.n) {
        gg = g.gid[i];
        if (dr.gs[gg].status == ST_RUNNING) {
            if (d > 0)
                bfs_vertex(g, dr, i, d);
            lv = dr.level[i];
            if (lv > h)
                lv = -1;
            if (lv >= 0)
                c = (unsigned int)(g.row_ptr[i + 1] - g.row_ptr[i]) * (lv == 0 ? 1u : 2u);
        }
    }
    // block-aggregated appends: per level, a warp ballot ranks the lanes, the
    // block's warps take consecutive ranges of one global reservation
    __shared__ int s_wcnt[LVL_MAX + 1][BLOCK / 32];
    __shared__ int s_base[LVL_MAX + 1];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int L = 0; L <= h; ++L) {
        const unsigned mask = __ballot_sync(0xffffffffu, lv == L);
        if (lane == 0)
            s_wcnt[L][warp] = __popc(mask);
    }
    __syncthreads();
    if (threadIdx.x <= (unsigned)h) {
        int tot = 0;
        for (int w = 0; w < BLOCK / 32; ++w)
            tot += s_wcnt[threadIdx.x][w];
        s_base[threadIdx.x] = tot ? atomicAdd(&dr.lvl_cnt[threadIdx.x], tot) : 0;
    }
    __syncthreads();
    for (int L = 0; L <= h; ++L) {
        const unsigned mask = __ballot_sync(0xffffffffu, lv == L);
        if (lv == L) {
            int before = s_base[L];
            for (unsigned w = 0; w < warp; ++w)
                before += s_wcnt[L][w];
            dr.lvl_list[(size_t)L * g.n + before + __popc(mask & ((1u << lane) - 1u))] = make_int2(i, g.row_ptr[i]);
        }
    }
    add_commit_counts(dr, uniform, g0, lv >= 0, gg, c, true);
}

// Residual Splash over the level lists, binary messages: commit of level Lc
// fused with the evaluation of level Le (the same sub-step pairing as
// k_splash_step), one thread per listed vertex, grid-stride.
template <typename S>
__global__ void __launch_bounds__(BLOCK, 6) k_splash_list_step(DevGraph g, DevRun dr, int Lc, int Le)
{
    griddep_launch_dependents();
    griddep_wait();
    const int nc = Lc >= 0 ? dr.lvl_cnt[Lc] : 0;
    const int ne = Le >= 0 ? dr.lvl_cnt[Le] : 0;
    const int2 *lc = dr.lvl_list + (size_t)(Lc >= 0 ? Lc : 0) * g.n;
    const int2 *le = dr.lvl_list + (size_t)(Le >= 0 ? Le : 0) * g.n;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc + ne; t += gridDim.x * blockDim.x) {
        if (t < nc) {
            const int2 vb = lc[t];
            splash_commit_vertex_b<S>(g, dr, vb.x, vb.y);
        } else {
            const int2 vb = le[t - nc];
            splash_eval_vertex_b<S, 4>(g, dr, vb.x, vb.y, Lc);
        }
    }
}

// --------------------------------------------------------------------------
// Set-up of a run.
template <typename S>
__global__ void k_init_msgs(S *a, S *b, size_t count, double value, float sc)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
         t += (size_t)gridDim.x * blockDim.x) {
        Store<S>::st(a + t, (typename Store<S>::A)value, sc);
        Store<S>::st(b + t, (typename Store<S>::A)value, sc);
    }
}

// Start messages of a k-state layout with absent states: a message into
// vertex j is uniform over j's present states and carries no mass (the log
// floor) on the absent ones.
template <typename S>
__global__ void k_init_msgs_var(DevGraph g, S *a, S *b)
{
    using A = typename Store<S>::A;
    const size_t count = (size_t)g.M * (size_t)g.k;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count; t += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(t / (size_t)g.k), x = (int)(t % (size_t)g.k);
        const int j = g.col[e];
        const bool present = !isinf(g.unary[(size_t)j * g.k + x]);
        const A v = present ? (A)(-log((double)g.kpresent[j])) : log_floor<A>();
        Store<S>::st(a + t, v, g.qscale);
        Store<S>::st(b + t, v, g.qscale);
    }
}

// --------------------------------------------------------------------------
// Binary Ising potentials (Eq. 1 with the coupling table of the Ising layout):
// validation and derived arrays on the device, so that setting the
// potentials of a large batch costs two copies and two passes.
// Checks: unary log-potentials finite (flags bit 0: NaN or +inf; bit 1: a
// vertex with both states -inf; bit 2: one state -inf, an absent state),
// couplings finite (bit 3) and symmetric, beta[rev e] == beta[e] (bit 4, the
// lowest such edge in bad_edge); max |beta| as float bits.
__global__ void k_pot_check_ising(const float *unary, const float *beta, const int32_t *rev, int n, int M,
                                  PotCheck *out)
{
    unsigned flags = 0, bmax = 0;
    int bad = 0x7fffffff;
    const int stride = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < max(n, M); t += stride) {
        if (t < n) {
            const float u0 = unary[2 * (size_t)t], u1 = unary[2 * (size_t)t + 1];
            if (isnan(u0) || isnan(u1) || (isinf(u0) && u0 > 0.0f) || (isinf(u1) && u1 > 0.0f))
                flags |= 1u;
            const int ninf = (isinf(u0) && u0 < 0.0f) + (isinf(u1) && u1 < 0.0f);
            flags |= ninf == 2 ? 2u : (ninf == 1 ? 4u : 0u);
        }
        if (t < M) {
            const float b = beta[t];
            if (!isfinite(b)) {
                flags |= 8u;
            } else {
                bmax = max(bmax, __float_as_uint(fabsf(b)));
                if (beta[rev[t]] != b) {
                    flags |= 16u;
                    bad = min(bad, t);
                }
            }
        }
    }
    flags = __reduce_or_sync(0xffffffffu, flags);
    bmax = __reduce_max_sync(0xffffffffu, bmax);
    bad = __reduce_min_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        if (flags)
            atomicOr(&out->flags, flags);
        if (bmax)
            atomicMax(&out->bmax_bits, bmax);
        if (bad != 0x7fffffff)
            atomicMin(&out->bad_edge, bad);
    }
}

// Derived arrays: udiff = u(1) - u(0) (FP64 and FP32), q = exp(-2 beta)
// clamped to [1e-300, 1e300] (FP64) and [1e-30, 1e30] (FP32). q32 holds beta
// on entry; each element is read and rewritten by the same thread.
__global__ void k_pot_derive_ising(const float *unary, float *q32, double *q64, float *ud32, double *ud64, int n,
                                   int M)
{
    const int stride = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < max(n, M); t += stride) {
        if (t < n) {
            const double d = (double)unary[2 * (size_t)t + 1] - (double)unary[2 * (size_t)t];
            ud64[t] = d;
            ud32[t] = (float)d;
        }
        if (t < M) {
            const double q = exp(-2.0 * (double)q32[t]);
            q64[t] = fmin(fmax(q, 1e-300), 1e300);
            q32[t] = (float)fmin(fmax(q, 1e-30), 1e30);
        }
    }
}

cudaError_t launch_pot_ising(const float *unary, float *beta_q32, double *q64, float *ud32, double *ud64,
                             const int32_t *rev, int n, int M, PotCheck *check, PotCheck *host_check)
{
    const int total = std::max(std::max(n, M), 1);
    const int nb = std::min((total + BLOCK - 1) / BLOCK, 152 * 16);
    cudaError_t e;
    PotCheck init;
    init.flags = 0;
    init.bad_edge = 0x7fffffff;
    init.bmax_bits = 0;
    init.pad = 0;
    if ((e = cudaMemcpy(check, &init, sizeof(PotCheck), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    k_pot_check_ising<<<nb, BLOCK>>>(unary, beta_q32, rev, n, M, check);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if ((e = cudaMemcpy(host_check, check, sizeof(PotCheck), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    if (host_check->flags)
        return cudaSuccess;   // the caller reports the first failed check; nothing derived
    k_pot_derive_ising<<<nb, BLOCK>>>(unary, beta_q32, q64, ud32, ud64, n, M);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return cudaDeviceSynchronize();
}

__global__ void k_init_state(DevRun dr, int G)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G * NSUB; t += gridDim.x * blockDim.x) {
        dr.red_max[t] = 0ull;
        dr.red_cnt[t] = 0u;
        if (dr.red_commit)
            dr.red_commit[t] = 0u;
        if (dr.red_commit_lo)
            dr.red_commit_lo[t] = 0u;
        if (t < G) {
            GState st;
            st.status = ST_RUNNING;
            st.rounds = 0;
            st.cur = 0;
            st.k_sel = 0;
            st.thr = 0;
            st.always = 0;
            st.n_prev = 0;
            st.committed = 0;
            st.evals = 0;
            st.full_evals = 0;
            st.full_nodes = 0;
            st.final_maxr = 0.0;
            st.final_cnt = 0;
            dr.gs[t] = st;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *dr.n_running = G;
        if (dr.queue)
            *dr.queue = 0;
    }
}

// Marks every still-running graph as stopped (wall-clock budget), folding the
// commits of its last round into its count.
__global__ void k_stop_running(DevRun dr, int G)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < G; t += gridDim.x * blockDim.x) {
        if (dr.gs[t].status == ST_RUNNING) {
            if (dr.red_commit) {
                unsigned long long c = 0;
                for (int q = 0; q < NSUB; ++q) {
                    c += dr.red_commit[(size_t)t * NSUB + q];
                    dr.red_commit[(size_t)t * NSUB + q] = 0u;
                }
                dr.gs[t].committed += c;
            }
            dr.gs[t].status = ST_STOPPED;
            atomicSub(dr.n_running, 1);
        }
    }
}

// --------------------------------------------------------------------------
// Beliefs (Eq. 3), normalised in FP64, and messages in the probability domain.
template <typename S>
__global__ void __launch_bounds__(BLOCK) k_beliefs_bin(DevGraph g, DevRun dr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n)
        return;
    const S *cur = (const S *)msg_buf(dr, dr.gs[g.gid[i]].cur);
    double h = g.udiff64[i];
    for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e)
        h += (double)Store<S>::ld(cur + g.rev[e], g.qscale);
    if constexpr (sizeof(typename Store<S>::A) == 8) {
        dr.beliefs[2 * (size_t)i + 1] = 1.0 / (1.0 + exp(-h));
        dr.beliefs[2 * (size_t)i] = 1.0 / (1.0 + exp(h));
    } else {
        // FP32 messages: exp in FP32 (relative error ~1e-7, below the
        // messages' own), the normalisation in FP64; e = exp(-|h|) <= 1
        const double e = (double)__expf(-(float)fabs(h));
        const double hi = 1.0 / (1.0 + e), lo = e / (1.0 + e);
        dr.beliefs[2 * (size_t)i + 1] = h >= 0.0 ? hi : lo;
        dr.beliefs[2 * (size_t)i] = h >= 0.0 ? lo : hi;
    }
}

template <typename S, int KP>
__global__ void __launch_bounds__(BLOCK) k_beliefs_gen(DevGraph g, DevRun dr)
{
    constexpr int NPB = BLOCK / KP;
    const int lane = threadIdx.x % KP;
    const int i = blockIdx.x * NPB + (int)threadIdx.x / KP;
    if (i >= g.n)
        return;
    const int k = g.k;
    const bool ok = lane < k;
    const S *cur = (const S *)msg_buf(dr, dr.gs[g.gid[i]].cur);
    double s = ok ? (double)g.unary[(size_t)i * k + lane] : -1e300;
    for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e)
        if (ok)
            s += (double)Store<S>::ld(cur + (size_t)g.rev[e] * k + lane, g.qscale);
    const unsigned gm = grp_mask<KP>();
    double mx = grp_max<KP>(gm, s);
    double w = ok ? exp(s - mx) : 0.0;
    double z = grp_sum<KP>(gm, w);
    if (ok)
        dr.beliefs[(size_t)i * k + lane] = w / z;
}

template <typename S>
__global__ void __launch_bounds__(BLOCK) k_messages_bin(DevGraph g, DevRun dr, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n)
        return;
    const S *cur = (const S *)msg_buf(dr, dr.gs[g.gid[i]].cur);
    for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
        double u = (double)Store<S>::ld(cur + e, g.qscale);
        out[2 * (size_t)e + 1] = 1.0 / (1.0 + exp(-u));
        out[2 * (size_t)e] = 1.0 / (1.0 + exp(u));
    }
}

template <typename S, int KP>
__global__ void __launch_bounds__(BLOCK) k_messages_gen(DevGraph g, DevRun dr, double *out)
{
    constexpr int NPB = BLOCK / KP;
    const int lane = threadIdx.x % KP;
    const int i = blockIdx.x * NPB + (int)threadIdx.x / KP;
    if (i >= g.n)
        return;
    const int k = g.k;
    const S *cur = (const S *)msg_buf(dr, dr.gs[g.gid[i]].cur);
    if (lane < k)
        for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e)
            out[(size_t)e * k + lane] = exp((double)Store<S>::ld(cur + (size_t)e * k + lane, g.qscale));
}

// --------------------------------------------------------------------------
// k-state messages with 32 < k <= 32 * SPL (the protein-folding graphs of
// Section IV-E reach 81 states): one warp per vertex, lane l holds states
// l, l + 32, ..., l + 32 (SPL - 1); the same Eq. 2 / Eq. 3 / Eq. 4 arithmetic
// as k_eval_gen, state by state. The shared table (k^2 floats, up to 64 KB)
// is read through the read-only cache instead of shared memory.
template <typename S, int SPL, int MODE>
__global__ void __launch_bounds__(BLOCK) k_eval_wide(DevGraph g, DevRun dr, RunParams rp, int level_L)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    const int k = g.k;
    constexpr int NPB = BLOCK / 32;
    const int lane = threadIdx.x & 31;
    const int first = blockIdx.x * NPB;
    const int last = min(g.n - 1, first + NPB - 1);
    const int g0 = g.gid[first];
    const bool uniform = (g0 == g.gid[last]);
    const int i = first + (int)threadIdx.x / 32;
    bool ok[SPL];
#pragma unroll
    for (int s = 0; s < SPL; ++s)
        ok[s] = lane + 32 * s < k;
    bool valid = false;
    int gg = g0;
    A maxa = 0;
    const A eps_a = eps_in(rp, (A)0);
    unsigned int cnt = 0;
    bool act = false;
    if (i < g.n) {
        gg = g.gid[i];
        act = dr.gs[gg].status == ST_RUNNING;
        if (MODE == MODE_SPLASH)
            act = act && (dr.level[i] == level_L);
    }
    if (act) {   // uniform across the warp
        valid = (lane == 0);
        const int cur_idx = dr.gs[gg].cur;
        const S *cur = (const S *)msg_buf(dr, cur_idx);
        S *out = (S *)msg_buf(dr, cur_idx ^ 1);
        const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
        A Sx[SPL];
#pragma unroll
        for (int s = 0; s < SPL; ++s)
            Sx[s] = ok[s] ? (A)g.unary[(size_t)i * k + lane + 32 * s] : (A)0;
        for (int e = beg; e < end; ++e) {
            const S *in = cur + (size_t)g.rev[e] * k + lane;
#pragma unroll
            for (int s = 0; s < SPL; ++s)
                if (ok[s])
                    Sx[s] += Store<S>::ld(in + 32 * s, g.qscale);
        }
        RT *R = (RT *)dr.resid;
        for (int e = beg; e < end; ++e) {
            const S *in = cur + (size_t)g.rev[e] * k + lane;
            A cav[SPL], a[SPL], acc[SPL];
            A mloc = (A)(-1e30);
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const A lin = ok[s] ? Store<S>::ld(in + 32 * s, g.qscale) : (A)0;
                cav[s] = ok[s] ? Sx[s] - lin : (A)(-1e30);
                mloc = cav[s] > mloc ? cav[s] : mloc;
            }
            const A mx = grp_max<32>(0xffffffffu, mloc);
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                a[s] = ok[s] ? m_exp(cav[s] - mx) : (A)0;
                acc[s] = 0;
            }
            const float *tab = g.pair + (size_t)e * k * k;
#pragma unroll
            for (int sx = 0; sx < SPL; ++sx) {
                for (int src = 0; src < 32; ++src) {
                    const int x = 32 * sx + src;
                    if (x >= k)
                        break;   // uniform across the warp
                    const A ax = __shfl_sync(0xffffffffu, a[sx], src);
#pragma unroll
                    for (int s = 0; s < SPL; ++s) {
                        if (!ok[s])
                            continue;
                        const int y = lane + 32 * s;
                        const A psi = g.pair_kind == 2 ? (A)__ldg(&g.psi_shared[x * k + y]) : m_exp((A)tab[x * k + y]);
                        acc[s] += ax * psi;
                    }
                }
            }
            A part = 0;
#pragma unroll
            for (int s = 0; s < SPL; ++s)
                part += ok[s] ? acc[s] : (A)0;
            const A z = grp_sum<32>(0xffffffffu, part);
            A lnew[SPL];
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                lnew[s] = ok[s] ? m_log(m_div(acc[s], z)) : (A)0;
                lnew[s] = lnew[s] > log_floor<A>() ? lnew[s] : log_floor<A>();
            }
            S *o = out + (size_t)e * k + lane;
            if (MODE == MODE_SPLASH) {
#pragma unroll
                for (int s = 0; s < SPL; ++s)
                    if (ok[s])
                        Store<S>::st(o + 32 * s, lnew[s], g.qscale);
                continue;
            }
            A rl = 0;
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                if (!ok[s])
                    continue;
                const A pn = m_exp(Store<S>::quant(lnew[s], g.qscale));
                const A po = m_exp(Store<S>::ld(cur + (size_t)e * k + lane + 32 * s, g.qscale));
                const A d = fabs(pn - po);
                rl = d > rl ? d : rl;
            }
            const A r = grp_max<32>(0xffffffffu, rl);
#pragma unroll
            for (int s = 0; s < SPL; ++s)
                if (ok[s])
                    Store<S>::st(o + 32 * s, lnew[s], g.qscale);
            if (MODE == MODE_CAND && lane == 0)
                R[e] = (RT)r;
            maxa = r > maxa ? r : maxa;
            cnt += (r >= eps_a) ? 1u : 0u;
        }
    }
    if (MODE != MODE_SPLASH)
        reduce_to_graph(dr, uniform, g0, valid, gg, (double)maxa, cnt);
}

// Beliefs (Eq. 3) and messages in the probability domain for 32 < k <= 32 SPL.
template <typename S, int SPL>
__global__ void __launch_bounds__(BLOCK) k_beliefs_wide(DevGraph g, DevRun dr)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (BLOCK / 32) + (int)threadIdx.x / 32;
    if (i >= g.n)
        return;
    const int k = g.k;
    const S *cur = (const S *)msg_buf(dr, dr.gs[g.gid[i]].cur);
    double sv[SPL];
    double mloc = -1e300;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
        const int x = lane + 32 * s;
        sv[s] = x < k ? (double)g.unary[(size_t)i * k + x] : -1e300;
        for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e)
            if (x < k)
                sv[s] += (double)Store<S>::ld(cur + (size_t)g.rev[e] * k + x, g.qscale);
        mloc = fmax(mloc, sv[s]);
    }
    const double mx = grp_max<32>(0xffffffffu, mloc);
    double w[SPL], part = 0.0;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
        w[s] = lane + 32 * s < k ? exp(sv[s] - mx) : 0.0;
        part += w[s];
    }
    const double z = grp_sum<32>(0xffffffffu, part);
#pragma unroll
    for (int s = 0; s < SPL; ++s)
        if (lane + 32 * s < k)
            dr.beliefs[(size_t)i * k + lane + 32 * s] = w[s] / z;
}

template <typename S, int SPL>
__global__ void __launch_bounds__(BLOCK) k_messages_wide(DevGraph g, DevRun dr, double *out)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (BLOCK / 32) + (int)threadIdx.x / 32;
    if (i >= g.n)
        return;
    const int k = g.k;
    const S *cur = (const S *)msg_buf(dr, dr.gs[g.gid[i]].cur);
    for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e)
#pragma unroll
        for (int s = 0; s < SPL; ++s)
            if (lane + 32 * s < k)
                out[(size_t)e * k + lane + 32 * s] =
                    exp((double)Store<S>::ld(cur + (size_t)e * k + lane + 32 * s, g.qscale));
}

// --------------------------------------------------------------------------
// Host-side launchers.
static inline int blocks_for(int n, int per_block) { return (n + per_block - 1) / per_block; }

// Launch of a kernel that calls griddep_wait before touching run state: with
// pdl, programmatic stream serialization lets its grid be scheduled while the
// previous kernel on the stream drains (in a captured graph the edge becomes
// a programmatic one); without it, an ordinary launch.
template <typename... KArgs, typename... Args>
static void launch_k(bool pdl, void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args... args)
{
    if (!pdl) {
        kernel<<<grid, block, 0, s>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)block, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Calls BODY with S bound to the storage type of dtype (Q16 only for the
// binary Ising layout, which the runtime enforces).
#define BPG_DISPATCH4(dtype, BODY)                                   \
    switch (dtype) {                                                 \
    case DT_F64: { using S = double; BODY; } break;                  \
    case DT_F32: { using S = float; BODY; } break;                   \
    case DT_BF16: { using S = __nv_bfloat16; BODY; } break;          \
    default: { using S = int16_t; BODY; } break;                     \
    }
#define BPG_DISPATCH3(dtype, BODY)                                   \
    switch (dtype) {                                                 \
    case DT_F64: { using S = double; BODY; } break;                  \
    case DT_F32: { using S = float; BODY; } break;                   \
    default: { using S = __nv_bfloat16; BODY; } break;               \
    }

template <typename S> constexpr int dtype_of()
{
    return sizeof(S) == 8 ? DT_F64 : (sizeof(S) == 4 ? DT_F32 : (std::is_same<S, int16_t>::value ? DT_Q16 : DT_BF16));
}

template <typename S>
static void launch_eval_bin(const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode, int level_L,
                            cudaStream_t s)
{
    int nb = blocks_for(g.n, BLOCK);
    (void)level_L;   // binary splash sweeps use k_splash_step / k_splash_list_step
    // mapping: thread per vertex (1), thread per vertex with the graph arrays
    // of 4 edges prefetched (4; 40 registers: 6 blocks per SM), streamed warp
    // tiles (6)
    if (rp.variant == 6) {
        launch_eval_stream(dtype_of<S>(), g, dr, rp, mode, s);
        return;
    }
    if (rp.variant == 4) {
        if (mode == MODE_LBP)
            launch_k(rp.pdl, k_eval_bin_pf<S, MODE_LBP, 4, 6>, nb, BLOCK, s, g, dr, rp);
        else
            launch_k(rp.pdl, k_eval_bin_pf<S, MODE_CAND, 4, 6>, nb, BLOCK, s, g, dr, rp);
        return;
    }
    if (mode == MODE_LBP)
        k_eval_bin<S, MODE_LBP><<<nb, BLOCK, 0, s>>>(g, dr, rp);
    else
        k_eval_bin<S, MODE_CAND><<<nb, BLOCK, 0, s>>>(g, dr, rp);
}

template <typename S, int KP>
static void launch_eval_gen(const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode, int level_L,
                            cudaStream_t s)
{
    int nb = blocks_for(g.n, BLOCK / KP);
    if (mode == MODE_LBP)
        k_eval_gen<S, KP, MODE_LBP><<<nb, BLOCK, 0, s>>>(g, dr, rp, level_L);
    else if (mode == MODE_CAND)
        k_eval_gen<S, KP, MODE_CAND><<<nb, BLOCK, 0, s>>>(g, dr, rp, level_L);
    else
        k_eval_gen<S, KP, MODE_SPLASH><<<nb, BLOCK, 0, s>>>(g, dr, rp, level_L);
}

void launch_eval(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode, int level_L,
                 int kp, cudaStream_t s)
{
    if (g.n == 0)
        return;
    if (g.epm == 1) {
        BPG_DISPATCH4(dtype, (launch_eval_bin<S>(g, dr, rp, mode, level_L, s)));
        return;
    }
    // (k-state messages use one KP-lane group per vertex)
    if (kp > 32) {
        // 32 < k <= 128: a warp per vertex, 2 or 4 states per lane
        const int nb = blocks_for(g.n, BLOCK / 32);
        auto go = [&](auto spl) {
            constexpr int SPL = decltype(spl)::value;
            BPG_DISPATCH3(dtype, (mode == MODE_LBP
                                      ? k_eval_wide<S, SPL, MODE_LBP><<<nb, BLOCK, 0, s>>>(g, dr, rp, level_L)
                                      : mode == MODE_CAND
                                            ? k_eval_wide<S, SPL, MODE_CAND><<<nb, BLOCK, 0, s>>>(g, dr, rp, level_L)
                                            : k_eval_wide<S, SPL, MODE_SPLASH><<<nb, BLOCK, 0, s>>>(g, dr, rp, level_L)))
        };
        if (kp == 64)
            go(std::integral_constant<int, 2>());
        else
            go(std::integral_constant<int, 4>());
    } else if (kp == 4)
        BPG_DISPATCH3(dtype, (launch_eval_gen<S, 4>(g, dr, rp, mode, level_L, s)))
    else if (kp == 8)
        BPG_DISPATCH3(dtype, (launch_eval_gen<S, 8>(g, dr, rp, mode, level_L, s)))
    else if (kp == 16)
        BPG_DISPATCH3(dtype, (launch_eval_gen<S, 16>(g, dr, rp, mode, level_L, s)))
    else
        BPG_DISPATCH3(dtype, (launch_eval_gen<S, 32>(g, dr, rp, mode, level_L, s)))
}

cudaError_t preload_lbp_f32_kernels()
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_eval_bin<float, MODE_LBP>);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, k_decide);
    if (e == cudaSuccess)
        e = cudaFuncGetAttributes(&fa, k_beliefs_bin<float>);
    return e;
}

void launch_decide(const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    const int per_block = DECIDE_BLOCK / 32;
    launch_k(rp.pdl, k_decide, (g.G + per_block - 1) / per_block, DECIDE_BLOCK, s, g, dr, rp);
}

void launch_commit_rnbp(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    if (g.n == 0)
        return;
    if (g.n_wtiles > 0 && rp.eps_words && g.epm == 1 && dtype != DT_F64) {
        // the flag words of the streamed update (FP32 / BF16 / Q16): one wave of lane groups
        auto go = [&](auto tag) {
            using S = decltype(tag);
            launch_k(rp.pdl, k_commit_rnbp_pipe<S>,
                     std::min(commit_pipe_blocks<S>(), blocks_for(g.n_wtiles, BLOCK / COMMIT_LPT)), BLOCK, s, g, dr,
                     rp);
        };
        if (dtype == DT_F32)
            go(float());
        else if (dtype == DT_BF16)
            go(__nv_bfloat16());
        else
            go(int16_t());
        return;
    }
    if (g.n_wtiles > 0) {
        // eight lanes per warp tile
        BPG_DISPATCH4(dtype, (launch_k(rp.pdl, k_commit_rnbp_wt<S>, blocks_for(g.n_wtiles, BLOCK / COMMIT_LPT), BLOCK, s,
                                       g, dr, rp)));
        return;
    }
    BPG_DISPATCH4(dtype, (launch_k(rp.pdl, k_commit_rnbp_tiled<S>, blocks_for(g.n, TILE_V), TILE_V, s, g, dr, rp)));
}

void launch_bfs_level(const DevGraph &g, const DevRun &dr, int d, cudaStream_t s)
{
    if (g.n == 0)
        return;
    k_bfs_level<<<blocks_for(g.n, BLOCK), BLOCK, 0, s>>>(g, dr, d);
}

void launch_bfs_level_lists(const DevGraph &g, const DevRun &dr, int d, int h, cudaStream_t s)
{
    if (g.n == 0)
        return;
    k_bfs_level_lists<<<blocks_for(g.n, BLOCK), BLOCK, 0, s>>>(g, dr, d, h);
}

void launch_splash_list_step(int dtype, const DevGraph &g, const DevRun &dr, int Lc, int Le, cudaStream_t s,
                             bool pdl)
{
    if (g.n == 0)
        return;
    const int nb = std::min(blocks_for(g.n, BLOCK), 152 * 6);   // one wave at 6 blocks per SM
    BPG_DISPATCH4(dtype, (launch_k(pdl, k_splash_list_step<S>, nb, BLOCK, s, g, dr, Lc, Le)));
}

void launch_splash_commit(int dtype, const DevGraph &g, const DevRun &dr, int level_L, cudaStream_t s)
{
    if (g.n == 0)
        return;
    int nb = blocks_for(g.n, BLOCK);
    BPG_DISPATCH4(dtype, (k_splash_commit<S><<<nb, BLOCK, 0, s>>>(g, dr, level_L)));
}

void launch_splash_step(int dtype, const DevGraph &g, const DevRun &dr, int Lc, int Le, cudaStream_t s)
{
    if (g.n == 0)
        return;
    int nb = blocks_for(g.n, BLOCK);
    BPG_DISPATCH4(dtype, (k_splash_step<S><<<nb, BLOCK, 0, s>>>(g, dr, Lc, Le)));
}

void launch_init(int dtype, const DevGraph &g, const DevRun &dr, cudaStream_t s)
{
    size_t count = (size_t)g.M * (size_t)g.epm;
    double v = (g.epm == 1) ? 0.0 : -log((double)g.k);
    if (count) {
        int nb = (int)std::min<size_t>((count + BLOCK - 1) / BLOCK, 152 * 16);
        if (g.epm > 1 && g.kpresent)
            BPG_DISPATCH3(dtype, (k_init_msgs_var<S><<<nb, BLOCK, 0, s>>>(g, (S *)dr.msg[0], (S *)dr.msg[1])))
        else
            BPG_DISPATCH4(dtype, (k_init_msgs<S><<<nb, BLOCK, 0, s>>>((S *)dr.msg[0], (S *)dr.msg[1], count, v,
                                                                      g.qscale)));
    }
    int nb2 = blocks_for(g.G * NSUB, BLOCK);
    k_init_state<<<nb2, BLOCK, 0, s>>>(dr, g.G);
}

void launch_stop_running(const DevGraph &g, const DevRun &dr, cudaStream_t s)
{
    k_stop_running<<<blocks_for(g.G, BLOCK), BLOCK, 0, s>>>(dr, g.G);
}

void launch_beliefs(int dtype, const DevGraph &g, const DevRun &dr, int kp, cudaStream_t s)
{
    if (g.n == 0)
        return;
    if (g.epm == 1) {
        int nb = blocks_for(g.n, BLOCK);
        BPG_DISPATCH4(dtype, (k_beliefs_bin<S><<<nb, BLOCK, 0, s>>>(g, dr)));
        return;
    }
    if (kp == 64)
        BPG_DISPATCH3(dtype, (k_beliefs_wide<S, 2><<<blocks_for(g.n, BLOCK / 32), BLOCK, 0, s>>>(g, dr)))
    else if (kp > 64)
        BPG_DISPATCH3(dtype, (k_beliefs_wide<S, 4><<<blocks_for(g.n, BLOCK / 32), BLOCK, 0, s>>>(g, dr)))
    else if (kp == 4)
        BPG_DISPATCH3(dtype, (k_beliefs_gen<S, 4><<<blocks_for(g.n, BLOCK / 4), BLOCK, 0, s>>>(g, dr)))
    else if (kp == 8)
        BPG_DISPATCH3(dtype, (k_beliefs_gen<S, 8><<<blocks_for(g.n, BLOCK / 8), BLOCK, 0, s>>>(g, dr)))
    else if (kp == 16)
        BPG_DISPATCH3(dtype, (k_beliefs_gen<S, 16><<<blocks_for(g.n, BLOCK / 16), BLOCK, 0, s>>>(g, dr)))
    else
        BPG_DISPATCH3(dtype, (k_beliefs_gen<S, 32><<<blocks_for(g.n, BLOCK / 32), BLOCK, 0, s>>>(g, dr)))
}

void launch_messages(int dtype, const DevGraph &g, const DevRun &dr, int kp, double *out, cudaStream_t s)
{
    if (g.n == 0)
        return;
    if (g.epm == 1) {
        int nb = blocks_for(g.n, BLOCK);
        BPG_DISPATCH4(dtype, (k_messages_bin<S><<<nb, BLOCK, 0, s>>>(g, dr, out)));
        return;
    }
    if (kp == 64)
        BPG_DISPATCH3(dtype, (k_messages_wide<S, 2><<<blocks_for(g.n, BLOCK / 32), BLOCK, 0, s>>>(g, dr, out)))
    else if (kp > 64)
        BPG_DISPATCH3(dtype, (k_messages_wide<S, 4><<<blocks_for(g.n, BLOCK / 32), BLOCK, 0, s>>>(g, dr, out)))
    else if (kp == 4)
        BPG_DISPATCH3(dtype, (k_messages_gen<S, 4><<<blocks_for(g.n, BLOCK / 4), BLOCK, 0, s>>>(g, dr, out)))
    else if (kp == 8)
        BPG_DISPATCH3(dtype, (k_messages_gen<S, 8><<<blocks_for(g.n, BLOCK / 8), BLOCK, 0, s>>>(g, dr, out)))
    else if (kp == 16)
        BPG_DISPATCH3(dtype, (k_messages_gen<S, 16><<<blocks_for(g.n, BLOCK / 16), BLOCK, 0, s>>>(g, dr, out)))
    else
        BPG_DISPATCH3(dtype, (k_messages_gen<S, 32><<<blocks_for(g.n, BLOCK / 32), BLOCK, 0, s>>>(g, dr, out)))
}

}  // namespace bpg
