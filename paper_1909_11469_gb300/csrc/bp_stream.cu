// Streamed warp-tile form of the binary Ising update (Eq. 2 in log-odds, the
// Eq. 4 residual and the per-graph convergence reduction fused), for the
// degree-irregular graphs where thread-per-vertex warps diverge and wait on
// long dependent load chains.
//
// The handle's vertices are cut into warp tiles: runs of consecutive vertices
// of one graph with at most WT out-edges and WV vertices (built on the host,
// int4 {first vertex, first edge, graph, vertex count} per tile plus a
// sentinel; a tile's edges end at the next record's first edge). A
// persistent grid deals the tiles to its warps round-robin. Each warp runs
// its own STAGES-deep pipeline: lane 0 streams a tile's contiguous arrays —
// rev, exp(-2 beta), the old messages, row_ptr and the unary log-odds — into
// the warp's shared memory with 1-D bulk copies (cp.async.bulk, completion on
// an mbarrier), STAGES - 1 tiles ahead of the one the warp computes. Per tile
// the lanes then
//   1. gather the incoming messages cur[rev[e]] (four independent loads per
//      lane, the only scattered accesses; a graph's messages sit in L2),
//   2. sum each vertex's field h_i = unary log-odds + incoming log-odds in
//      edge order (one lane per vertex, from shared memory),
//   3. form every out-message from the cavity h_i - u_{j->i}, its residual,
//      and store both coalesced.
// The arithmetic and its order are those of the per-vertex routine, so every
// mapping writes the same bits.
#include "bp_internal.cuh"
#include "bp_launch.h"

#include <algorithm>
#include <mutex>

namespace bpg {

namespace {

constexpr int SW_WARPS = 8;                      // warps per block
constexpr int SW_THREADS = 32 * SW_WARPS;
constexpr int SW_STAGES = 3;                     // tiles in flight per warp
constexpr long long SW_WAIT_LIMIT = 1ll << 22;   // bounded mbarrier polls

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

constexpr int round16(int b) { return (b + 15) & ~15; }

// Shared-memory layout of one warp, in bytes.
template <typename S> struct SwLayout {
    static constexpr int REV = (STREAM_WT + 8) * 4;                    // rev, reused for the gathered u_in
    static constexpr int Q = (STREAM_WT + 8) * 4;                      // exp(-2 beta)
    static constexpr int OLD = round16((STREAM_WT + 16) * (int)sizeof(S));   // stored messages
    static constexpr int RP = (STREAM_WV + 8) * 4;                     // row_ptr
    static constexpr int UD = (STREAM_WV + 8) * 4;                     // unary log-odds
    static constexpr int STAGE = REV + Q + OLD + RP + UD;
    static constexpr int MBAR = 0;                                     // SW_STAGES x 8 bytes
    static constexpr int INFO = 64;                                    // SW_STAGES x 8 ints
    static constexpr int H = INFO + SW_STAGES * 32;                    // STREAM_WV floats
    static constexpr int SRC = H + STREAM_WV * 4;                      // STREAM_WT bytes
    static constexpr int STAGES0 = (SRC + STREAM_WT + 127) / 128 * 128;   // 128-byte aligned stages
    static constexpr int WARP = (STAGES0 + SW_STAGES * STAGE + 127) / 128 * 128;
};

__device__ __forceinline__ void mbar_init(unsigned a, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// One bounded poll loop on phase `parity` of the barrier; false when the
// limit ran out.
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

// Per-stage record written by lane 0 when it issues a tile.
struct SwInfo {
    int v0, e0, v1, e1, g, cur, valid, pad;
};

// (max residual, count) of one graph from every lane of the warp into a
// reduction sub-slot.
template <typename A>
__device__ __forceinline__ void sw_flush(const DevRun &dr, int gg, A maxa, unsigned cnt, int slot)
{
    unsigned long long mb = (unsigned long long)__double_as_longlong((double)maxa);
    mb = warp_max_u64(mb);
    cnt = warp_sum_u32(cnt);
    if ((threadIdx.x & 31) == 0 && gg >= 0) {
        if (mb)
            atomicMax(&dr.red_max[(size_t)gg * NSUB + slot], mb);
        if (cnt)
            atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], cnt);
    }
}

template <typename S, int MODE>
__global__ void __launch_bounds__(SW_THREADS) k_eval_bin_stream(DevGraph g, DevRun dr, RunParams rp)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    using L = SwLayout<S>;
    static_assert(sizeof(A) == 4, "FP32 arithmetic only");
    extern __shared__ __align__(128) unsigned char sw_raw[];
    griddep_launch_dependents();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *wbase = sw_raw + (size_t)warp * L::WARP;
    SwInfo *info = reinterpret_cast<SwInfo *>(wbase + L::INFO);
    A *s_h = reinterpret_cast<A *>(wbase + L::H);
    uint8_t *s_src = wbase + L::SRC;
    const unsigned mbar0 = smem_addr(wbase + L::MBAR);
    if (lane == 0) {
        for (int s = 0; s < SW_STAGES; ++s)
            mbar_init(mbar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // Tiles are dealt round-robin: warp gw takes tiles gw, gw + W, gw + 2W, ...
    // (W = warps of the grid), so the warps of the grid sweep the arrays
    // together and the graphs being gathered at any time stay few (their
    // messages in L2). j counts the warp's own tiles.
    const int nt = g.n_wtiles;
    const int gw = blockIdx.x * SW_WARPS + warp;
    const int wtot = gridDim.x * SW_WARPS;
    const int n_local = gw < nt ? (nt - gw + wtot - 1) / wtot : 0;
    const int slot = gw & (NSUB - 1);
    const float qs = g.qscale;
    const A *qarr = (const A *)g.q32;
    RT *R = (RT *)dr.resid;
    // the graph arrays are constant during a run; the run state (graph status,
    // message buffers) is read only after the previous kernel has finished
    griddep_wait();

    // Window of tile records for the issuing side: lane l holds the warp's
    // tile jb + l (first vertex and edge, its end, its graph and that graph's state).
    int jb = -64;
    int w_v0 = 0, w_e0 = 0, w_v1 = 0, w_e1 = 0, w_g = 0, w_run = 0, w_cur = 0;
    auto load_window = [&](int base) {
        jb = base;
        const int jl = base + lane;
        const int t = gw + jl * wtot;
        w_run = 0;
        if (jl < n_local) {
            const int4 a = g.wtiles[t];
            w_v0 = a.x;
            w_e0 = a.y;
            w_g = a.z;
            w_v1 = a.x + a.w;
            w_e1 = g.wtiles[t + 1].y;
            const GState *st = dr.gs + w_g;
            w_run = st->status == ST_RUNNING;
            w_cur = st->cur;
        }
    };
    // Issues the warp's tile j into stage s (every lane calls it; lane 0 copies).
    auto issue = [&](int j, int s) {
        if (j >= n_local) {
            if (lane == 0)
                info[s].valid = 0;
            return;
        }
        if (j >= jb + 32)
            load_window(j);
        const int src = j - jb;
        const int v0 = __shfl_sync(0xffffffffu, w_v0, src);
        const int e0 = __shfl_sync(0xffffffffu, w_e0, src);
        const int v1 = __shfl_sync(0xffffffffu, w_v1, src);
        const int e1 = __shfl_sync(0xffffffffu, w_e1, src);
        const int gg = __shfl_sync(0xffffffffu, w_g, src);
        const int run = __shfl_sync(0xffffffffu, w_run, src);
        const int cb = __shfl_sync(0xffffffffu, w_cur, src);
        if (lane == 0) {
            SwInfo &in = info[s];
            in.v0 = v0;
            in.e0 = e0;
            in.v1 = v1;
            in.e1 = e1;
            in.g = gg;
            in.cur = cb;
            in.valid = run;
            if (run) {
                constexpr int EPS = 16 / (int)sizeof(S);   // stored elements per 16 bytes
                const int e0a = e0 & ~3, e0s = e0 & ~(EPS - 1), v0a = v0 & ~3;
                const unsigned b_rev = (unsigned)round16((e1 - e0a) * 4);
                const unsigned b_old = (unsigned)round16((e1 - e0s) * (int)sizeof(S));
                const unsigned b_rp = (unsigned)round16((v1 + 1 - v0a) * 4);
                const unsigned b_ud = (unsigned)round16((v1 - v0a) * 4);
                const unsigned mb = mbar0 + 8 * s;
                const unsigned st0 = smem_addr(wbase + L::STAGES0 + s * L::STAGE);
                mbar_expect_tx(mb, 2 * b_rev + b_old + b_rp + b_ud);
                const S *cur = (const S *)msg_buf(dr, cb);
                bulk_load(st0, g.rev + e0a, b_rev, mb);
                bulk_load(st0 + L::REV, qarr + e0a, b_rev, mb);
                bulk_load(st0 + L::REV + L::Q, cur + e0s, b_old, mb);
                bulk_load(st0 + L::REV + L::Q + L::OLD, g.row_ptr + v0a, b_rp, mb);
                bulk_load(st0 + L::REV + L::Q + L::OLD + L::RP, g.udiff32 + v0a, b_ud, mb);
            }
        }
    };

    for (int s = 0; s < SW_STAGES; ++s)
        issue(s, s);
    __syncwarp();

    unsigned phase = 0;   // bit s: parity of stage s's next completion
    int acc_g = -1;
    A maxa = 0;
    unsigned cnt = 0;
    const A eps_a = eps_in(rp, (A)0);
    bool failed = false;
    for (int j = 0; j < n_local; ++j) {
        const int s = j % SW_STAGES;
        const SwInfo in = info[s];
        if (in.valid) {
            const unsigned mb = mbar0 + 8 * s;
            if (!mbar_wait_bounded(mb, (phase >> s) & 1u)) {
                failed = true;
                break;
            }
            phase ^= 1u << s;
            if (in.g != acc_g) {
                sw_flush(dr, acc_g, maxa, cnt, slot);
                acc_g = in.g;
                maxa = 0;
                cnt = 0;
            }
            constexpr int EPS = 16 / (int)sizeof(S);
            unsigned char *st = wbase + L::STAGES0 + s * L::STAGE;
            int *s_rev = reinterpret_cast<int *>(st);
            A *s_uin = reinterpret_cast<A *>(st);
            const A *s_q = reinterpret_cast<const A *>(st + L::REV);
            const S *s_old = reinterpret_cast<const S *>(st + L::REV + L::Q);
            const int *s_rp = reinterpret_cast<const int *>(st + L::REV + L::Q + L::OLD);
            const A *s_ud = reinterpret_cast<const A *>(st + L::REV + L::Q + L::OLD + L::RP);
            const int ro = in.e0 - (in.e0 & ~3);
            const int oo = in.e0 - (in.e0 & ~(EPS - 1));
            const int vo = in.v0 - (in.v0 & ~3);
            const int ne = in.e1 - in.e0, nv = in.v1 - in.v0;
            const S *cur = (const S *)msg_buf(dr, in.cur);
            S *out = (S *)msg_buf(dr, in.cur ^ 1);
            // 1. incoming messages
            constexpr int EPL = STREAM_WT / 32;
            A uin[EPL];
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const int idx = lane + 32 * k;
                if (idx < ne)
                    uin[k] = Store<S>::ld(cur + s_rev[ro + idx], qs);
            }
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const int idx = lane + 32 * k;
                if (idx < ne)
                    s_uin[ro + idx] = uin[k];
            }
            __syncwarp();
            // 2. vertex fields, in edge order
            if (lane < nv) {
                const int b = s_rp[vo + lane] - in.e0, en = s_rp[vo + lane + 1] - in.e0;
                A h = s_ud[vo + lane];
                for (int x = b; x < en; ++x) {
                    h += s_uin[ro + x];
                    s_src[x] = (uint8_t)lane;
                }
                s_h[lane] = h;
            }
            __syncwarp();
            // 3. out-messages, residuals
#pragma unroll
            for (int k = 0; k < EPL; ++k) {
                const int idx = lane + 32 * k;
                if (idx < ne) {
                    const int e = in.e0 + idx;
                    const A unew = ising_logodds(s_q[ro + idx], s_h[s_src[idx]] - uin[k]);
                    const A uq = Store<S>::quant(unew, qs);
                    const A r = fabs(m_sigmoid(uq) - m_sigmoid(Store<S>::val(s_old[oo + idx], qs)));
                    Store<S>::st(out + e, unew, qs);
                    if (MODE == MODE_CAND)
                        R[e] = (RT)r;
                    maxa = r > maxa ? r : maxa;
                    cnt += (r >= eps_a) ? 1u : 0u;
                }
            }
        }
        // the stage's shared memory is free again: order the lanes' reads and
        // writes of it before the bulk copy that refills it
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(j + SW_STAGES, s);
        __syncwarp();
    }
    if (failed) {
        // a completion wait ran out: record it, let the copies this warp has
        // in flight land (bounded), and leave
        if (lane == 0)
            atomicExch(dr.err, 1);
        for (int s = 0; s < SW_STAGES; ++s)
            if (info[s].valid)
                mbar_wait_bounded(mbar0 + 8 * s, (phase >> s) & 1u);
        return;
    }
    sw_flush(dr, acc_g, maxa, cnt, slot);
}

template <typename S> constexpr int sw_smem_bytes() { return SW_WARPS * SwLayout<S>::WARP; }

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
    // at least ~2 tiles per warp, at most one wave of resident blocks
    const int want = (g.n_wtiles + 2 * SW_WARPS - 1) / (2 * SW_WARPS);
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
}

void launch_eval_stream(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode,
                        cudaStream_t s)
{
    if (g.n_wtiles == 0)
        return;
    const bool cand = mode != MODE_LBP;
    switch (dtype) {
    case DT_F32:
        cand ? launch_stream_t<float, MODE_CAND>(g, dr, rp, s) : launch_stream_t<float, MODE_LBP>(g, dr, rp, s);
        break;
    case DT_BF16:
        cand ? launch_stream_t<__nv_bfloat16, MODE_CAND>(g, dr, rp, s)
             : launch_stream_t<__nv_bfloat16, MODE_LBP>(g, dr, rp, s);
        break;
    default:
        cand ? launch_stream_t<int16_t, MODE_CAND>(g, dr, rp, s) : launch_stream_t<int16_t, MODE_LBP>(g, dr, rp, s);
        break;
    }
}

}  // namespace bpg
