// Internal device structures and helpers of libbp_gb300 (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bpg {

// Per-graph run status.
enum : int32_t { ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAXROUNDS = 2, ST_STOPPED = 3 };

// Sub-slots per graph for the max/count reductions (spreads same-address atomics).
constexpr int NSUB = 32;

// Per-graph device state, one per graph of a handle.
struct GState {
    int32_t status;
    int32_t rounds;        // committing rounds so far
    int32_t cur;           // message buffer holding the committed state
    int32_t k_sel;         // RBP/RS frontier size of the current round
    uint32_t thr;          // RnBP threshold floor(p * 2^16) of the current round
    int32_t always;        // RnBP: p >= 1 this round
    uint64_t n_prev;       // RnBP: unconverged count of the previous round
    unsigned long long committed;
    unsigned long long evals;        // all message evaluations (full + splash)
    unsigned long long full_evals;   // messages evaluated by full-evaluation launches
    unsigned long long full_nodes;   // vertices processed by full-evaluation launches
    double final_maxr;
    unsigned long long final_cnt;
};

// Warp tiles of the streamed update (bp_stream.cu): at most STREAM_WT
// out-edges and STREAM_WV consecutive vertices of one graph.
constexpr int STREAM_WT = 128;
constexpr int STREAM_WV = 32;

// Read-only graph and potential arrays on the device.
struct DevGraph {
    int32_t n, k, G;
    int32_t M;
    int32_t epm;              // stored elements per message: 1 (binary log-odds) or k
    float qscale;             // scale of the run's 16-bit storage: Q16 log-odds per integer
                              // step; BF16 binary log-odds per unit of log2 of the stored
                              // word; 0 for BF16 k-state logs (plain rounding)
    int32_t vec_ok;           // 1: rev, q and message buffers are 16-byte aligned
    int32_t sel_smem_bytes;   // dynamic shared memory of the selection kernels (set per launch)
    int32_t max_ge;           // largest directed-edge count of a graph
    int32_t max_gv;           // largest vertex count of a graph
    int32_t sel_c[2];         // selection clusters: CTAs per graph (RBP, RS), planned per run
    int32_t sel_dyn[2];       // selection clusters: staged-key bytes per CTA (RBP, RS)
    int32_t sel_grid[2];      // 1: select with the grid-wide kernels instead (RBP, RS)
    const int32_t *row_ptr;   // [n+1]
    const int32_t *col;       // [M]
    const int32_t *rev;       // [M]
    const int32_t *gid;       // [n] graph of each vertex
    const int32_t *gv_off;    // [G+1]
    const int32_t *ge_off;    // [G+1]
    // potentials
    int32_t pair_kind;
    const float *unary;       // [n*k] log-potentials
    const float *udiff32;     // [n]  theta_i(1) - theta_i(0)      (k = 2, Ising)
    const double *udiff64;    // [n]
    const float *q32;         // [M]  exp(-2 beta_e)                (k = 2, Ising)
    const double *q64;        // [M]
    const float *pair;        // table [M*k*k] (log) or shared [k*k] (log)
    const float *psi_shared;  // [k*k] exp(Theta - max Theta)     (shared)
    const int32_t *kpresent;  // [n] present states per vertex (unary > -inf), or null when all k are
    // streamed update: warp tiles {first vertex, first edge, graph, vertex
    // count}, every vertex in one tile, and a sentinel {n, M, -1, 0};
    // n_wtiles = 0 when a vertex has > STREAM_WT edges
    const int4 *wtiles;
    int32_t n_wtiles;
    // per warp tile {first edge, end edge, graph, graph's first edge} (the
    // RnBP commit's record: no dependent graph-offset load)
    const int4 *ctiles;
};

// Per-run parameters (kernel arguments, baked into the captured graph).
struct RunParams {
    int32_t schedule;
    int32_t max_rounds;
    double eps;
    double low_p;
    double high_p;
    double ratio_threshold;
    uint64_t seed;
    uint32_t graph_id_base;
    int32_t splash_depth;
    int32_t rs_roots_mode;
    int32_t record_trace;
    int32_t trace_capacity;
    int32_t trace_words;      // words per recorded round
    int32_t variant;          // binary update mapping: 1 thread per vertex, 2 tiled edge quads
    float eps_f;              // smallest float >= eps: (double)r >= eps  <=>  r >= eps_f for float r
    int32_t tc_path;          // shared-table update: 0 per-vertex, 1 tiles/CUDA cores, 2 tiles/tensor
                              // cores, 3 tiles/tensor cores with residual products
    int32_t sel_grid;         // grid-wide selection: bit 0 RBP, bit 1 RS (keys the captured rounds)
    int32_t pdl;              // 1: the update, decision and RnBP commit kernels are launched
                              // with programmatic stream serialization
    int32_t dynamic_p;        // 1: RBP / RS frontier fraction switched per round by EdgeRatio
    int32_t eps_words;        // 1: the streamed update writes the eps flag words (DevRun::eps_words)
                              // and the RnBP commit reads them instead of the residuals
    int32_t fused_rnbp;       // 1: RnBP rounds commit inside the streamed update (three message
                              // buffers, GState::cur in 0..2), no commit kernel
};

// eps in the residual type, chosen so that the comparison equals the FP64 test.
__device__ __forceinline__ float eps_in(const RunParams &rp, float) { return rp.eps_f; }
__device__ __forceinline__ double eps_in(const RunParams &rp, double) { return rp.eps; }

// Grid-wide selection state of one graph (large graphs, bp_select_grid.cu):
// the key prefix fixed so far (the threshold after the last pass), the rank
// of the k-th key inside the current digit (after the last pass: the number of
// threshold ties to take) and the count of keys in that digit.
struct GSelState {
    unsigned long long prefix;
    int32_t krem;
    int32_t eq_total;
};

// Mutable per-run device buffers.
struct DevRun {
    void *msg[3];                 // message buffers (storage dtype); the third only for the fused
                                  // RnBP rounds
    void *resid;                  // [M] residuals (float, or double for FP64)
    void *vres;                   // [n] vertex residuals for RS (residual type)
    int8_t *level;                // [n] splash level (-1 none)
    GState *gs;                   // [G]
    unsigned long long *red_max;  // [G*NSUB] double bits
    unsigned int *red_cnt;        // [G*NSUB]
    unsigned int *red_commit;     // [G*NSUB] RnBP commits of the round per sub-slot, folded into
                                  // GState::committed by the next decision (null: not used); with
                                  // the fused RnBP rounds, the commits of the HighP outcome
    unsigned int *red_commit_lo;  // [G*NSUB] fused RnBP rounds: the commits of the LowP outcome
    int32_t *n_running;           // [1]
    uint32_t *trace;              // [trace_capacity * trace_words]
    double *beliefs;              // [n*k]
    int32_t *queue;               // [1] next graph for the persistent batch kernel
    int2 *lvl_list;               // [(LVL_MAX+1) * n] Residual Splash vertices of each level:
                                  // (vertex, its first out-edge)
    int32_t *lvl_cnt;             // [LVL_MAX+1] entries of each level list
    const double *graph_p;        // [G] per-graph parallelism, or null: every graph uses rp.low_p
    int32_t *err;                 // [1] set when a bounded device wait runs out
    uint32_t *eps_words;          // [4 n_wtiles] per warp tile of the streamed update: bit i of
                                  // word w = message e0 + 32 w + i has residual >= eps
    // grid-wide selection (large graphs; null when unused)
    GSelState *gsel;              // [G]
    unsigned int *gsel_hist;      // [G * 2048]
    int32_t *gsel_tie;            // [chunks] threshold ties per chunk, then their exclusive scan
    const int32_t *chunk_off;     // [2 (G + 1)] chunk offsets per graph: RBP (edges), then RS (vertices)
    int32_t n_chunks_rbp, n_chunks_rs;
};

// Parallelism of graph gg: RnBP LowP, or the RBP / RS frontier fraction.
__device__ __forceinline__ double graph_low_p(const DevRun &dr, const RunParams &rp, int gg)
{
    return dr.graph_p ? dr.graph_p[gg] : rp.low_p;
}

// EdgeRatio switch of Section IV-A for committing round `rounds` (1-based)
// with n_now messages of residual >= eps now and n_prev at the previous
// evaluation: HighP in round 1, then LowP when n_now / n_prev > the threshold
// (bad convergence), else HighP. RnBP uses it every round; RBP and RS use it
// with dynamic_p for their frontier fraction.
__device__ __forceinline__ bool edge_ratio_low(const RunParams &rp, int rounds, unsigned long long n_now,
                                               unsigned long long n_prev)
{
    return rounds != 1 && (double)n_now / (double)n_prev > rp.ratio_threshold;
}
__device__ __forceinline__ double edge_ratio_p(const RunParams &rp, double low_p, int rounds,
                                               unsigned long long n_now, unsigned long long n_prev)
{
    return edge_ratio_low(rp, rounds, n_now, n_prev) ? low_p : rp.high_p;
}

// RnBP random-filter threshold of frontier probability p (R7: a 16-bit draw
// is kept when below floor(p 2^16)); p >= 1 keeps every eligible message.
__device__ __forceinline__ void rnbp_threshold(double p, uint32_t &thr, int &always)
{
    always = (p >= 1.0) ? 1 : 0;
    thr = (p <= 0.0 || p >= 1.0) ? 0u : (uint32_t)(p * 65536.0);
}

// Programmatic dependent launch: a grid launched with programmatic stream
// serialization may start while its predecessor on the stream finishes; this
// waits until every prerequisite grid has completed and its memory is
// visible. In a grid launched without that attribute it returns at once.
// Every thread of such a grid calls it before its first access to data that
// a kernel of the run writes.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next grid on the stream (when launched with that attribute) be
// scheduled once every block of this grid has executed it; that grid still
// waits for this one's completion in griddep_wait. A no-op otherwise.
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }

// Deepest splash whose sweeps run over per-level vertex lists (binary messages).
constexpr int LVL_MAX = 3;

// Message buffer b (0 or 1). A select instead of msg[b]: indexing the kernel
// parameter array with a runtime value would copy the whole struct to local memory.
__device__ __forceinline__ void *msg_buf(const DevRun &dr, int b) { return dr.msg[b]; }

// ---------------------------------------------------------------------------
// Storage traits: message element type S, arithmetic type A. sc is the Q16
// step (log-odds per integer unit); the floating formats ignore it.
template <typename S> struct Store;
template <> struct Store<double> {
    using A = double;
    static __device__ __forceinline__ double ld(const double *p, float) { return *p; }
    static __device__ __forceinline__ double val(double x, float) { return x; }
    static __device__ __forceinline__ void st(double *p, double v, float) { *p = v; }
    static __device__ __forceinline__ double quant(double v, float) { return v; }
};
template <> struct Store<float> {
    using A = float;
    static __device__ __forceinline__ float ld(const float *p, float) { return *p; }
    static __device__ __forceinline__ float val(float x, float) { return x; }
    static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
    static __device__ __forceinline__ float quant(float v, float) { return v; }
};
// BF16. With sc > 0 (binary Ising log-odds; sc a power of two) the word is
// the bfloat16 value nearest to w = 2^(|u| / sc - 125), carrying the sign of u:
// for |u| <= 250 sc it lies in [2^-125, 2^125], and its exponent and mantissa
// bits form a logarithmic code of |u| with a step of at most sc / 128; read
// back as |u| = (log2 |w| + 125) sc. With sc = 0 (k-state logs) the word is the
// value itself rounded to bfloat16. ex2 / lg2 are the hardware approximations,
// the scaling by sc and 1/sc is exact, so every kernel codes and decodes the
// same bits.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> struct Store<__nv_bfloat16> {
    using A = float;
    static __device__ __forceinline__ __nv_bfloat16 code(float v, float sc)
    {
        if (sc <= 0.0f)
            return __float2bfloat16_rn(v);
        const float inv = __int_as_float(0x7F000000 - __float_as_int(sc));   // 1 / sc, exact for a power of two
        const float w = ex2_approx(__fsub_rn(__fmul_rn(fabsf(v), inv), 125.0f));
        return __float2bfloat16_rn(v < 0.0f ? -w : w);
    }
    static __device__ __forceinline__ float val(__nv_bfloat16 x, float sc)
    {
        const float w = __bfloat162float(x);
        if (sc <= 0.0f)
            return w;
        const float a = __fmul_rn(__fadd_rn(lg2_approx(fabsf(w)), 125.0f), sc);
        return w < 0.0f ? -a : a;
    }
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, float sc) { return val(*p, sc); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, float sc) { *p = code(v, sc); }
    static __device__ __forceinline__ float quant(float v, float sc) { return val(code(v, sc), sc); }
};
// Q16: binary log-odds as a signed 16-bit multiple of sc, |q| <= 32767. The
// products q * sc are rounded explicitly (__fmul_rn), so no kernel fuses them
// into a neighbouring addition and every kernel decodes the same value.
template <> struct Store<int16_t> {
    using A = float;
    static __device__ __forceinline__ float code(float v, float sc)
    {
        float q = rintf(__fdividef(v, sc));
        return fminf(fmaxf(q, -32767.0f), 32767.0f);
    }
    static __device__ __forceinline__ float ld(const int16_t *p, float sc) { return __fmul_rn((float)*p, sc); }
    static __device__ __forceinline__ float val(int16_t x, float sc) { return __fmul_rn((float)x, sc); }
    static __device__ __forceinline__ void st(int16_t *p, float v, float sc) { *p = (int16_t)code(v, sc); }
    static __device__ __forceinline__ float quant(float v, float sc) { return __fmul_rn(code(v, sc), sc); }
};

// Residual element type: double for FP64 messages, float otherwise.
template <typename S> struct ResidT { using T = float; };
template <> struct ResidT<double> { using T = double; };

// ---------------------------------------------------------------------------
// Math in the arithmetic type. FP32 uses the SFU intrinsics.
__device__ __forceinline__ float m_exp(float x) { return __expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_log(float x) { return __logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ float m_sigmoid(float u) { return __fdividef(1.0f, 1.0f + __expf(-u)); }
__device__ __forceinline__ double m_sigmoid(double u) { return 1.0 / (1.0 + exp(-u)); }

// Binary Ising message in log-odds u = log m(1) - log m(0).
// With cavity log-odds h of x_i and q = exp(-2 beta):
//   u = sign(h) * log((1 + q F) / (q + F)),  F = exp(-|h|),
// which is log[(e^{-b} + e^{b+h}) / (e^{b} + e^{h-b})] rearranged so that no
// term overflows (the sum over x_i of Eq. 2 for the 2x2 Ising table). The
// product q F is rounded explicitly (fmaf / __dmul_rn), so every kernel that
// inlines this computes the same bits whatever the compiler contracts around it.
__device__ __forceinline__ float ising_logodds(float q, float h)
{
    float F = __expf(-fabsf(h));
    float u = __logf(__fdividef(fmaf(q, F, 1.0f), q + F));
    return h >= 0.0f ? u : -u;
}
__device__ __forceinline__ double ising_logodds(double q, double h)
{
    double F = exp(-fabs(h));
    double u = log1p(__dmul_rn(q, F)) - log(q + F);
    return h >= 0.0 ? u : -u;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), one block of four words.
__device__ __forceinline__ uint4 philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                         uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// RnBP random filter (Section IV-A): the Philox block of key seed and counter
// (local_edge / 8, round, graph id, 0) serves eight consecutive messages of a
// graph; message local_edge draws the 16-bit half (local_edge mod 2: 0 low,
// 1 high) of word (local_edge mod 8) / 2 and is selected when the half is
// below the round's threshold floor(p 2^16).
constexpr int RNBP_PER_BLOCK = 8;
__device__ __forceinline__ uint4 rnbp_block(const RunParams &rp, uint32_t octet, uint32_t round, uint32_t graph)
{
    return philox4(octet, round, rp.graph_id_base + graph, 0u, (uint32_t)(rp.seed & 0xffffffffu),
                   (uint32_t)(rp.seed >> 32));
}
__device__ __forceinline__ uint32_t rnbp_draw16(const uint4 &b, uint32_t j)
{
    const uint32_t w = j < 2 ? b.x : (j < 4 ? b.y : (j < 6 ? b.z : b.w));
    return (j & 1u) ? (w >> 16) : (w & 0xffffu);
}
__device__ __forceinline__ bool rnbp_pick(const RunParams &rp, uint32_t local_edge, uint32_t round,
                                          uint32_t graph, const GState &st)
{
    if (st.always)
        return true;
    return rnbp_draw16(rnbp_block(rp, local_edge >> 3, round, graph), local_edge & 7u) < st.thr;
}

// ---------------------------------------------------------------------------
// Reductions of (max residual, count >= eps) into per-graph sub-slots.
// Threads of a block cover consecutive vertices, so graph ids are monotone
// within a block; a block whose first and last vertex share a graph reduces
// in shared memory and issues one atomic per quantity.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned int warp_sum_u32(unsigned int v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// All threads of the block must call this. g = graph of the thread's item (any
// value if !valid); uniform = block-wide flag that every valid item has graph g0.
__device__ __forceinline__ void reduce_to_graph(const DevRun &dr, bool uniform, int32_t g0,
                                                bool valid, int32_t g, double maxr, unsigned int cnt)
{
    unsigned long long mb = valid ? (unsigned long long)__double_as_longlong(maxr) : 0ull;
    unsigned int c = valid ? cnt : 0u;
    int slot = blockIdx.x & (NSUB - 1);
    if (uniform) {
        __shared__ unsigned long long s_max[32];
        __shared__ unsigned int s_cnt[32];
        mb = warp_max_u64(mb);
        c = warp_sum_u32(c);
        int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) {
            s_max[warp] = mb;
            s_cnt[warp] = c;
        }
        __syncthreads();
        if (warp == 0) {
            int nw = (blockDim.x + 31) >> 5;
            mb = lane < nw ? s_max[lane] : 0ull;
            c = lane < nw ? s_cnt[lane] : 0u;
            mb = warp_max_u64(mb);
            c = warp_sum_u32(c);
            if (lane == 0) {
                if (mb)
                    atomicMax(&dr.red_max[(size_t)g0 * NSUB + slot], mb);
                if (c)
                    atomicAdd(&dr.red_cnt[(size_t)g0 * NSUB + slot], c);
            }
        }
    } else if (valid) {
        if (mb)
            atomicMax(&dr.red_max[(size_t)g * NSUB + slot], mb);
        if (c)
            atomicAdd(&dr.red_cnt[(size_t)g * NSUB + slot], c);
    }
}

}  // namespace bpg
