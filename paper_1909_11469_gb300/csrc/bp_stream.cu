// Streamed tile form of the binary Ising update (Eq. 2 in log-odds, the
// Eq. 4 residual and the per-graph convergence reduction fused), for the
// degree-irregular graphs where thread-per-vertex warps diverge and wait on
// long dependent load chains.
//
// The handle's vertices are cut into warp tiles: runs of consecutive vertices
// of one graph with at most STREAM_WT out-edges and STREAM_WV vertices (built
// on the host: int4 {first vertex, first edge, graph, vertex count} per tile,
// every vertex in exactly one tile, plus a sentinel; a tile ends where the
// next begins). Sixteen consecutive warp tiles form a block tile, whose edges and
// vertices are contiguous. A persistent grid deals the block tiles to its
// blocks round-robin, so the grid sweeps the arrays together and the graphs
// being gathered at any time stay few (their messages in L2).
//
// In each block one producer warp streams a block tile's arrays — rev,
// exp(-2 beta), the old messages, row_ptr and the unary log-odds — into a
// STAGES-deep ring of shared-memory stages with 1-D bulk copies (cp.async.bulk,
// completion on a "full" mbarrier), refilling a stage once its consumers have
// released it (an "empty" mbarrier). Each of the sixteen consumer warps takes one
// warp tile of the stage:
//   1. gather the incoming messages cur[rev[e]] (four independent loads per
//      lane, the only scattered accesses),
//   2. sum each vertex's field h_i = unary log-odds + incoming log-odds in
//      edge order (one lane per vertex, from shared memory),
//   3. form every out-message from the cavity h_i - u_{j->i}, its residual,
//      and store both coalesced.
// The arithmetic and its order are those of the per-vertex routine, so every
// mapping writes the same bits. Every wait is bounded: on expiry the kernel
// sets an error flag that the host reports.
//
// RnBP rounds can commit inside this kernel (MODE_RNBP_FUSED). The round's
// frontier probability is LowP or HighP, chosen by EdgeRatio from this
// round's count of messages with residual >= eps, which is known only after
// the whole graph is evaluated. The update therefore writes both outcomes:
// a message is kept in an outcome when it passes the eps test and its 16-bit
// Philox draw (R7) is below that outcome's threshold, and the outcome then
// holds the new message, else the old stored word. With the committed
// messages in buffer c of three, HighP goes to buffer c + 1 and LowP to
// c + 2 (mod 3); the decision moves the graph to the chosen one. Each tile's
// 8-message Philox blocks are drawn by one lane each (<= 17 per tile) while
// the gathers are in flight, and handed to the message lanes through shared
// memory: the block's four words read as eight little-endian 16-bit halves
// are the draws of its eight messages in order (half j = draw j of R7).
// This replaces the copying commit kernel, which touched nearly every sector
// of two buffers (~40% of messages selected), with one more coalesced
// stream of stores.
#include "bp_internal.cuh"
#include "bp_launch.h"

#include <algorithm>
#include <mutex>

namespace bpg {

namespace {

constexpr int SW_CONSUMERS = 16;                       // consumer warps (warp tiles per block tile)
constexpr int SW_THREADS = 32 * (SW_CONSUMERS + 1);    // + the producer warp
constexpr int SW_STAGES = 2;                           // block tiles in flight per block
// (16 consumers and 2 stages measured faster than 8 and 3 on the 4096-graph
// ER batch: 98 / 107 us per LBP / RnBP update against 101 / 115; the smaller
// ring leaves room for more resident warps)
constexpr int SW_BE = SW_CONSUMERS * STREAM_WT;        // edges per block tile (at most)
constexpr int SW_BV = SW_CONSUMERS * STREAM_WV;        // vertices per block tile (at most)
constexpr long long SW_WAIT_LIMIT = 1ll << 22;         // bounded mbarrier polls

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

constexpr int round16(int b) { return (b + 15) & ~15; }

// Per-stage record of a block tile, written by the producer's lane 0.
struct SwInfo {
    int valid;             // some warp tile of the block tile belongs to a running graph
    int cur;               // message buffer of the running graphs
    int e0a, e0s, v0a;     // first elements of the staged edge, message and vertex arrays
    int v0[SW_CONSUMERS + 1], e0[SW_CONSUMERS + 1], g[SW_CONSUMERS], run[SW_CONSUMERS];
    // fused RnBP rounds, per warp tile: the graph's committed buffer, its
    // completed rounds, its first edge and its LowP draw threshold (65536:
    // every eligible message)
    int cb[SW_CONSUMERS], rnd[SW_CONSUMERS], ge0[SW_CONSUMERS];
    unsigned tlo[SW_CONSUMERS];
};

// Shared-memory layout, in bytes.
template <typename S> struct SwLayout {
    static constexpr int REV = (SW_BE + 8) * 4;                          // rev, reused for the gathered u_in
    static constexpr int Q = (SW_BE + 8) * 4;                            // exp(-2 beta)
    static constexpr int OLD = round16((SW_BE + 16) * (int)sizeof(S));   // stored messages
    static constexpr int RP = (SW_BV + 8) * 4;                           // row_ptr
    static constexpr int UD = (SW_BV + 8) * 4;                           // unary log-odds
    static constexpr int STAGE = REV + Q + OLD + RP + UD;
    static constexpr int FULL = 0;                                       // SW_STAGES x 8 bytes
    static constexpr int EMPTY = 64;                                     // SW_STAGES x 8 bytes
    static constexpr int INFO = 128;                                     // SW_STAGES records
    static constexpr int WARPS = round16(INFO + SW_STAGES * (int)sizeof(SwInfo));
    // per consumer: h, src, and (fused RnBP rounds) the tile's Philox blocks,
    // read back as 16-bit draws (<= 17 blocks of 16 bytes)
    static constexpr int DRAW = STREAM_WV * 4 + STREAM_WT;
    static constexpr int WARP_B = DRAW + 18 * 16;
    static constexpr int STAGES0 = (WARPS + SW_CONSUMERS * WARP_B + 127) / 128 * 128;
    static constexpr int TOTAL = STAGES0 + SW_STAGES * STAGE;
};

__device__ __forceinline__ void mbar_init(unsigned a, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// Bounded poll loop on phase `parity` of the barrier; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned a, unsigned parity)
{
    for (long long it = 0; it < SW_WAIT_LIMIT; ++it) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done)
            return true;
    }
    return false;
}
// 1-D bulk copy global -> this CTA's shared memory; both addresses 16-byte
// aligned, bytes a multiple of 16; completion counted on the barrier.
__device__ __forceinline__ void bulk_load(unsigned dst, const void *src, unsigned bytes, unsigned mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// (max residual, count) of one graph from every lane of a warp into a
// reduction sub-slot. The residuals are non-negative floats, whose bit
// patterns order like the values, so the warp max is one integer reduction.
// With the fused RnBP rounds also the commits of the HighP and LowP outcomes.
template <bool FUSED>
__device__ __forceinline__ void sw_flush(const DevRun &dr, int gg, float maxa, unsigned cnt, unsigned chi,
                                         unsigned clo, int slot)
{
    const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(maxa));
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (FUSED) {
        chi = __reduce_add_sync(0xffffffffu, chi);
        clo = __reduce_add_sync(0xffffffffu, clo);
    }
    if ((threadIdx.x & 31) == 0 && gg >= 0) {
        if (mb)
            atomicMax(&dr.red_max[(size_t)gg * NSUB + slot],
                      (unsigned long long)__double_as_longlong((double)__uint_as_float(mb)));
        if (cnt)
            atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], cnt);
        if (FUSED && chi)
            atomicAdd(&dr.red_commit[(size_t)gg * NSUB + slot], chi);
        if (FUSED && clo)
            atomicAdd(&dr.red_commit_lo[(size_t)gg * NSUB + slot], clo);
    }
}

// Draw threshold of frontier probability p for the fused RnBP rounds: the
// R7 threshold, or 65536 (above every 16-bit draw) when p >= 1.
__device__ __forceinline__ unsigned sw_draw_threshold(double p)
{
    uint32_t thr;
    int always;
    rnbp_threshold(p, thr, always);
    return always ? 65536u : thr;
}

template <typename S, int MODE>
__global__ void __launch_bounds__(SW_THREADS, MODE == MODE_RNBP_FUSED ? 2 : 1)
    k_eval_bin_stream(DevGraph g, DevRun dr, RunParams rp)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    using L = SwLayout<S>;
    constexpr bool FUSED = MODE == MODE_RNBP_FUSED;
    static_assert(sizeof(A) == 4, "FP32 arithmetic only");
    constexpr int EPS = 16 / (int)sizeof(S);   // stored message elements per 16 bytes
    extern __shared__ __align__(128) unsigned char sw_raw[];
    griddep_launch_dependents();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    SwInfo *info = reinterpret_cast<SwInfo *>(sw_raw + L::INFO);
    const unsigned full0 = smem_addr(sw_raw + L::FULL), empty0 = smem_addr(sw_raw + L::EMPTY);
    if (threadIdx.x == 0) {
        for (int s = 0; s < SW_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, SW_CONSUMERS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int nwt = g.n_wtiles;
    const int nbt = (nwt + SW_CONSUMERS - 1) / SW_CONSUMERS;           // block tiles
    const int n_local = (int)blockIdx.x < nbt ? (nbt - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    // the graph arrays are constant during a run; the run state (graph status,
    // message buffers) is read only after the previous kernel has finished
    griddep_wait();

    if (warp == 0) {
        // ---------------- producer
        for (int i = 0; i < n_local; ++i) {
            const int s = i % SW_STAGES;
            if (i >= SW_STAGES && !mbar_wait_bounded(empty0 + 8 * s, ((i / SW_STAGES) - 1) & 1)) {
                if (lane == 0)
                    atomicExch(dr.err, 1);
                return;
            }
            const int bt = (int)blockIdx.x + i * (int)gridDim.x;
            const int t = bt * SW_CONSUMERS + lane;   // lanes 0..8: the records of the block tile
            int v0 = 0, e0 = 0, gg = -1, run = 0, cb = 0, rnd = 0, ge0 = 0;
            unsigned tlo = 0;
            if (lane <= SW_CONSUMERS && t <= nwt) {
                const int4 r = g.wtiles[t];
                v0 = r.x;
                e0 = r.y;
                gg = r.z;
            }
            if (lane < SW_CONSUMERS && t < nwt) {
                const GState *st = dr.gs + gg;
                run = st->status == ST_RUNNING;
                cb = st->cur;
                if (FUSED) {
                    rnd = st->rounds;
                    ge0 = g.ge_off[gg];
                    tlo = sw_draw_threshold(graph_low_p(dr, rp, gg));
                }
            }
            const int last = min(SW_CONSUMERS, nwt - bt * SW_CONSUMERS);   // warp tiles in this block tile
            const int v_end = __shfl_sync(0xffffffffu, v0, last);
            const int e_end = __shfl_sync(0xffffffffu, e0, last);
            // a warp tile without edges has nothing to update
            const int e_next = __shfl_down_sync(0xffffffffu, e0, 1);
            run = run && e_next > e0;
            const unsigned runm = __ballot_sync(0xffffffffu, run != 0) & ((1u << SW_CONSUMERS) - 1u);
            const int cur = runm ? __shfl_sync(0xffffffffu, cb, __ffs(runm) - 1) : 0;
            const int v_beg = __shfl_sync(0xffffffffu, v0, 0);
            const int e_beg = __shfl_sync(0xffffffffu, e0, 0);
            SwInfo &in = info[s];
            if (lane <= SW_CONSUMERS) {
                in.v0[lane] = v0;
                in.e0[lane] = e0;
            }
            if (lane < SW_CONSUMERS) {
                in.g[lane] = gg;
                in.run[lane] = (lane < last) && run;
                if (FUSED) {
                    in.cb[lane] = cb;
                    in.rnd[lane] = rnd;
                    in.ge0[lane] = ge0;
                    in.tlo[lane] = tlo;
                }
            }
            __syncwarp();
            if (lane == 0) {
                in.valid = runm != 0;
                in.cur = cur;
                const int e0a = e_beg & ~3, e0s = e_beg & ~(EPS - 1), v0a = v_beg & ~3;
                in.e0a = e0a;
                in.e0s = e0s;
                in.v0a = v0a;
                const unsigned mb = full0 + 8 * s;
                if (runm) {
                    // (the fused RnBP tiles read their old messages from their own graph's buffer)
                    const unsigned b_rev = (unsigned)round16((e_end - e0a) * 4);
                    const unsigned b_old = FUSED ? 0u : (unsigned)round16((e_end - e0s) * (int)sizeof(S));
                    const unsigned b_rp = (unsigned)round16((v_end + 1 - v0a) * 4);
                    const unsigned b_ud = (unsigned)round16((v_end - v0a) * 4);
                    const unsigned st0 = smem_addr(sw_raw + L::STAGES0 + s * L::STAGE);
                    mbar_expect_tx(mb, 2 * b_rev + b_old + b_rp + b_ud);
                    bulk_load(st0, g.rev + e0a, b_rev, mb);
                    bulk_load(st0 + L::REV, (const A *)g.q32 + e0a, b_rev, mb);
                    if (!FUSED)
                        bulk_load(st0 + L::REV + L::Q, (const S *)msg_buf(dr, cur) + e0s, b_old, mb);
                    bulk_load(st0 + L::REV + L::Q + L::OLD, g.row_ptr + v0a, b_rp, mb);
                    bulk_load(st0 + L::REV + L::Q + L::OLD + L::RP, g.udiff32 + v0a, b_ud, mb);
                } else {
                    mbar_arrive(mb);   // nothing to stream: complete the phase for the consumers
                }
            }
            __syncwarp();
        }
        return;
    }

    // ---------------- consumers
    const int c = warp - 1;
    unsigned char *wb = sw_raw + L::WARPS + c * L::WARP_B;
    A *s_h = reinterpret_cast<A *>(wb);
    uint8_t *s_src = wb + STREAM_WV * 4;
    uint4 *s_draw = reinterpret_cast<uint4 *>(wb + L::DRAW);
    const int slot = ((int)blockIdx.x * SW_CONSUMERS + c) & (NSUB - 1);
    const float qs = g.qscale;
    RT *R = (RT *)dr.resid;
    const A eps_a = eps_in(rp, (A)0);
    int acc_g = -1;
    A maxa = 0;
    unsigned cnt = 0, chi = 0, clo = 0;
    const unsigned thi = FUSED ? sw_draw_threshold(rp.high_p) : 0u;
    for (int i = 0; i < n_local; ++i) {
        const int s = i % SW_STAGES;
        if (!mbar_wait_bounded(full0 + 8 * s, (i / SW_STAGES) & 1)) {
            if (lane == 0)
                atomicExch(dr.err, 1);
            return;
        }
        const SwInfo &in = info[s];
        if (in.valid && in.run[c]) {
            const int v0 = in.v0[c], e0 = in.e0[c];
            const int nv = in.v0[c + 1] - v0, ne = in.e0[c + 1] - e0;
            const int gg = in.g[c];
            if (gg != acc_g) {
                sw_flush<FUSED>(dr, acc_g, maxa, cnt, chi, clo, slot);
                acc_g = gg;
                maxa = 0;
                cnt = 0;
                chi = 0;
                clo = 0;
            }
            unsigned char *st = sw_raw + L::STAGES0 + s * L::STAGE;
            const int ro = e0 - in.e0a, oo = e0 - in.e0s, vo = v0 - in.v0a;
            int *s_rev = reinterpret_cast<int *>(st) + ro;
            A *s_uin = reinterpret_cast<A *>(st) + ro;
            const A *s_q = reinterpret_cast<const A *>(st + L::REV) + ro;
            const S *s_old = reinterpret_cast<const S *>(st + L::REV + L::Q) + oo;
            const int *s_rp = reinterpret_cast<const int *>(st + L::REV + L::Q + L::OLD) + vo;
            const A *s_ud = reinterpret_cast<const A *>(st + L::REV + L::Q + L::OLD + L::RP) + vo;
            const int cbuf = FUSED ? in.cb[c] : in.cur;
            const S *cur = (const S *)msg_buf(dr, cbuf);
            S *out = (S *)msg_buf(dr, FUSED ? (cbuf == 2 ? 0 : cbuf + 1) : (cbuf ^ 1));   // (fused: HighP)
            S *out_lo = (S *)msg_buf(dr, FUSED ? (cbuf == 0 ? 2 : cbuf - 1) : 0);        // (fused: LowP)
            // 1. incoming messages (fused: and the tile's own old messages)
            constexpr int EPL = STREAM_WT / 32;
            A uin[EPL];
            S oldw[EPL];
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const int idx = lane + 32 * k;
                if (idx < ne) {
                    uin[k] = Store<S>::ld(cur + s_rev[idx], qs);
                    if (FUSED)
                        oldw[k] = cur[e0 + idx];
                }
            }
            // fused: the tile's Philox blocks, one per lane, while the loads are
            // in flight (octet j of the graph's messages holds local messages
            // 8 j .. 8 j + 7; the tile starts at local message m0)
            int off = 0;
            unsigned tlo = 0;
            bool draws = false;
            if (FUSED) {
                tlo = in.tlo[c];
                draws = !(tlo == 65536u && thi == 65536u);
                const int m0 = e0 - in.ge0[c];
                off = m0 & 7;
                if (draws && lane < ((off + ne + 7) >> 3))
                    s_draw[lane] = rnbp_block(rp, (uint32_t)((m0 >> 3) + lane), (uint32_t)(in.rnd[c] + 1), (uint32_t)gg);
            }
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const int idx = lane + 32 * k;
                if (idx < ne)
                    s_uin[idx] = uin[k];
            }
            __syncwarp();
            // 2. vertex fields, in edge order
            if (lane < nv) {
                const int b = s_rp[lane] - e0, en = s_rp[lane + 1] - e0;
                A h = s_ud[lane];
                for (int x = b; x < en; ++x) {
                    h += s_uin[x];
                    s_src[x] = (uint8_t)lane;
                }
                s_h[lane] = h;
            }
            __syncwarp();
            // 3. out-messages, residuals
            const size_t wt = ((size_t)blockIdx.x + (size_t)i * gridDim.x) * SW_CONSUMERS + c;   // warp tile
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const int idx = lane + 32 * k;
                bool hit = false;
                if (idx < ne) {
                    const int e = e0 + idx;
                    const A unew = ising_logodds(s_q[idx], s_h[s_src[idx]] - uin[k]);
                    const A uq = Store<S>::quant(unew, qs);
                    const A r = fabs(m_sigmoid(uq) - m_sigmoid(Store<S>::val(FUSED ? oldw[k] : s_old[idx], qs)));
                    if (MODE == MODE_CAND || FUSED)
                        R[e] = (RT)r;
                    maxa = r > maxa ? r : maxa;
                    hit = r >= eps_a;
                    cnt += hit ? 1u : 0u;
                    if constexpr (FUSED) {
                        // this message's 16-bit draw (tile message idx is draw idx + off
                        // of the tile's first block); both outcomes: the new message
                        // where kept, else the old stored word
                        const unsigned u = draws ? (unsigned)reinterpret_cast<const uint16_t *>(s_draw)[idx + off] : 0u;
                        const bool phi = hit && u < thi, plo = hit && u < tlo;
                        if (phi)
                            Store<S>::st(out + e, unew, qs);
                        else
                            out[e] = oldw[k];
                        if (plo)
                            Store<S>::st(out_lo + e, unew, qs);
                        else
                            out_lo[e] = oldw[k];
                        chi += phi ? 1u : 0u;
                        clo += plo ? 1u : 0u;
                    } else {
                        Store<S>::st(out + e, unew, qs);
                    }
                }
                if (MODE == MODE_CAND && rp.eps_words) {
                    // the eps test of 32 consecutive messages of the tile, for the RnBP commit
                    const unsigned w = __ballot_sync(0xffffffffu, hit);
                    if (lane == 0)
                        dr.eps_words[wt * 4 + k] = w;
                }
            }
        }
        // release the stage: order this warp's shared-memory accesses of it
        // (generic proxy) before the bulk copy that will refill it (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0)
            mbar_arrive(empty0 + 8 * s);
    }
    sw_flush<FUSED>(dr, acc_g, maxa, cnt, chi, clo, slot);
}

template <typename S> constexpr int sw_smem_bytes() { return SwLayout<S>::TOTAL; }

template <typename S, int MODE> int sw_blocks_per_sm()
{
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    std::call_once(once[dev], [&] {
        cudaFuncSetAttribute(k_eval_bin_stream<S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sw_smem_bytes<S>());
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval_bin_stream<S, MODE>, SW_THREADS,
                                                          sw_smem_bytes<S>()) != cudaSuccess)
            nb = 1;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = std::max(nb, 1) * std::max(sms, 1);
    });
    return cached[dev];
}

template <typename S, int MODE> void launch_stream_t(const DevGraph &g, const DevRun &dr, const RunParams &rp,
                                                     cudaStream_t s)
{
    const int max_blocks = sw_blocks_per_sm<S, MODE>();
    // at least ~2 block tiles per block, at most one wave of resident blocks
    const int want = (g.n_wtiles + 2 * SW_CONSUMERS - 1) / (2 * SW_CONSUMERS);
    const int grid = std::max(1, std::min(max_blocks, want));
    if (!rp.pdl) {
        k_eval_bin_stream<S, MODE><<<grid, SW_THREADS, sw_smem_bytes<S>(), s>>>(g, dr, rp);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(SW_THREADS, 1, 1);
    cfg.dynamicSmemBytes = sw_smem_bytes<S>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_eval_bin_stream<S, MODE>, g, dr, rp);
}

}  // namespace

void prepare_stream_kernels()
{
    sw_blocks_per_sm<float, MODE_LBP>();
    sw_blocks_per_sm<float, MODE_CAND>();
    sw_blocks_per_sm<__nv_bfloat16, MODE_LBP>();
    sw_blocks_per_sm<__nv_bfloat16, MODE_CAND>();
    sw_blocks_per_sm<int16_t, MODE_LBP>();
    sw_blocks_per_sm<int16_t, MODE_CAND>();
    sw_blocks_per_sm<float, MODE_RNBP_FUSED>();
    sw_blocks_per_sm<__nv_bfloat16, MODE_RNBP_FUSED>();
    sw_blocks_per_sm<int16_t, MODE_RNBP_FUSED>();
}

void launch_eval_stream(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode,
                        cudaStream_t s)
{
    if (g.n_wtiles == 0)
        return;
    auto go = [&](auto tag) {
        using S = decltype(tag);
        if (mode == MODE_LBP)
            launch_stream_t<S, MODE_LBP>(g, dr, rp, s);
        else if (mode == MODE_RNBP_FUSED)
            launch_stream_t<S, MODE_RNBP_FUSED>(g, dr, rp, s);
        else
            launch_stream_t<S, MODE_CAND>(g, dr, rp, s);
    };
    switch (dtype) {
    case DT_F32:
        go(float());
        break;
    case DT_BF16:
        go(__nv_bfloat16());
        break;
    default:
        go(int16_t());
        break;
    }
}

}  // namespace bpg
