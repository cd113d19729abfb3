// Frontier selection for Residual BP and Residual Splash on large graphs
// (Section III-D): the same exact top-k (ties to the smaller id) as the
// cluster kernels of bp_select.cu, spread over the whole GPU.
//
// A cluster owns at most 8 SMs, so a graph of millions of messages would be
// selected by 8 SMs while 144 idle. For a handful of large graphs the radix
// select runs as a sequence of grid-wide kernels instead:
//   hist   every block histograms a contiguous range of keys (11-bit digit)
//          in shared memory and adds the non-zero bins to its graph's global
//          histogram; keys whose higher digits differ from the graph's prefix
//          are skipped
//   digit  one block per graph scans the histogram from the top, fixes the
//          digit holding the k-th key and clears the histogram
// (three rounds of both for 32-bit keys, six for 64-bit ones), then
//   ties   per chunk of a graph, the keys equal to the threshold, and a scan
//          of those counts per graph (only when the ties straddle the
//          threshold; otherwise both exit at once)
//   apply  takes every key above the threshold and the lowest-id ties: RBP
//          commits the candidate message, RS marks the splash roots.
// RS first forms the vertex residuals (max over incoming messages, pull form).
#include "bp_internal.cuh"
#include "bp_launch.h"

#include <algorithm>

namespace bpg {

constexpr int GS_THREADS = 512;
constexpr int GS_BINS = 2048;
constexpr int GS_CHUNK = 2048;   // keys per apply block (4 per thread)

__device__ __forceinline__ uint32_t gkey(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long gkey(double v) { return (unsigned long long)__double_as_longlong(v); }

// Digit layout of pass p: 32-bit keys 11/11/10 bits, 64-bit keys 11 x 5 + 9.
template <typename KeyT> struct Digits;
template <> struct Digits<uint32_t> {
    static constexpr int passes = 3;
    static __host__ __device__ int shift(int p) { return p == 0 ? 21 : (p == 1 ? 10 : 0); }
    static __host__ __device__ int width(int p) { return p == 2 ? 10 : 11; }
};
template <> struct Digits<unsigned long long> {
    static constexpr int passes = 6;
    static __host__ __device__ int shift(int p) { return p < 5 ? 53 - 11 * p : 0; }
    static __host__ __device__ int width(int p) { return p < 5 ? 11 : 9; }
};

// Graph of key index x (keys of graph q are [off[q], off[q+1])), by binary
// search over the G + 1 offsets.
__device__ __forceinline__ int graph_of(const int32_t *off, int G, int x)
{
    int lo = 0, hi = G;   // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Key of index x: RBP the message residual, RS the vertex residual.
template <typename RT, bool RS>
__device__ __forceinline__ auto key_at(const DevRun &dr, int x)
{
    const RT *R = RS ? (const RT *)dr.vres : (const RT *)dr.resid;
    return gkey(R[x]);
}

// RS: vertex residual = max residual of the messages into the vertex (pull:
// vertex v gathers R[rev[e]] over its row), for vertices of running graphs.
template <typename RT>
__global__ void __launch_bounds__(GS_THREADS) k_gsel_vres(DevGraph g, DevRun dr)
{
    const RT *R = (const RT *)dr.resid;
    RT *V = (RT *)dr.vres;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x) {
        if (dr.gs[g.gid[v]].status != ST_RUNNING)
            continue;
        RT m = 0;
        for (int e = g.row_ptr[v]; e < g.row_ptr[v + 1]; ++e) {
            const RT r = R[g.rev[e]];
            m = r > m ? r : m;
        }
        V[v] = m;
    }
}

// Start of a selection: prefix 0, k = the round's frontier size.
__global__ void k_gsel_init(DevGraph g, DevRun dr)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.G; q += gridDim.x * blockDim.x) {
        GSelState s;
        s.prefix = 0ull;
        s.krem = dr.gs[q].k_sel;
        s.eq_total = 0;
        dr.gsel[q] = s;
    }
}

template <typename RT, bool RS>
__global__ void __launch_bounds__(GS_THREADS) k_gsel_hist(DevGraph g, DevRun dr, int pass)
{
    using KeyT = decltype(gkey((RT)0));
    using D = Digits<KeyT>;
    __shared__ unsigned int h[GS_BINS];
    const int32_t *off = RS ? g.gv_off : g.ge_off;
    const int total = RS ? g.n : (int)g.M;
    const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
    const int x0 = min(total, (int)blockIdx.x * per), x1 = min(total, x0 + per);
    if (x0 >= x1)
        return;
    const int gb = graph_of(off, g.G, x0);   // the block's (first) graph: shared-memory bins
    for (int t = threadIdx.x; t < GS_BINS; t += blockDim.x)
        h[t] = 0u;
    __syncthreads();
    const int shift = D::shift(pass), width = D::width(pass);
    const KeyT dmask = ((KeyT)1 << width) - 1;
    const int hs = shift + width;   // bits at and above hs are fixed by earlier passes
    int gcur = gb;
    bool run = dr.gs[gb].status == ST_RUNNING;
    KeyT pre = run ? (KeyT)dr.gsel[gb].prefix : 0;
    for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
        if (x >= off[gcur + 1] || x < off[gcur]) {
            gcur = graph_of(off, g.G, x);
            run = dr.gs[gcur].status == ST_RUNNING;
            pre = run ? (KeyT)dr.gsel[gcur].prefix : 0;
        }
        if (!run)
            continue;
        const KeyT k = key_at<RT, RS>(dr, x);
        if (hs < (int)(8 * sizeof(KeyT)) && (k >> hs) != (pre >> hs))
            continue;
        const unsigned d = (unsigned)((k >> shift) & dmask);
        if (gcur == gb)
            atomicAdd(&h[d], 1u);
        else
            atomicAdd(&dr.gsel_hist[(size_t)gcur * GS_BINS + d], 1u);
    }
    __syncthreads();
    if (dr.gs[gb].status != ST_RUNNING)
        return;
    for (int t = threadIdx.x; t < GS_BINS; t += blockDim.x)
        if (h[t])
            atomicAdd(&dr.gsel_hist[(size_t)gb * GS_BINS + t], h[t]);
}

// One block of 1024 threads per graph: digit of the krem-th largest key.
template <typename RT>
__global__ void __launch_bounds__(1024) k_gsel_digit(DevGraph g, DevRun dr, int pass)
{
    using KeyT = decltype(gkey((RT)0));
    using D = Digits<KeyT>;
    __shared__ unsigned int warp_tot[32];
    __shared__ unsigned int warp_excl[32];
    const int q = blockIdx.x;
    if (dr.gs[q].status != ST_RUNNING)
        return;
    unsigned int *hist = dr.gsel_hist + (size_t)q * GS_BINS;
    const int nb = 1 << D::width(pass);
    const int per = nb / (int)blockDim.x;   // 2, 1 (11 / 10 bits); 9 bits: 0 or 1 for half the threads
    const int krem = dr.gsel[q].krem;
    // thread t owns bins from the top: t * per .. t * per + per - 1 (descending digits)
    unsigned v[2] = {0u, 0u};
    unsigned mine = 0;
    const int own = per > 0 ? per : ((int)threadIdx.x < nb ? 1 : 0);
    for (int j = 0; j < own; ++j) {
        const int d = nb - 1 - ((int)threadIdx.x * (per > 0 ? per : 1) + j);
        v[j] = hist[d];
        mine += v[j];
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
        warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += y;
        }
        warp_excl[lane] = wi - w;
    }
    __syncthreads();
    incl += warp_excl[warp];
    unsigned acc = incl - mine;
    if (own > 0 && acc < (unsigned)krem && (unsigned)krem <= incl) {
        for (int j = 0; j < own; ++j) {
            if (acc + v[j] >= (unsigned)krem) {
                const int d = nb - 1 - ((int)threadIdx.x * (per > 0 ? per : 1) + j);
                GSelState s = dr.gsel[q];
                s.prefix = (unsigned long long)((KeyT)s.prefix | ((KeyT)d << D::shift(pass)));
                s.krem = krem - (int)acc;
                s.eq_total = (int)v[j];
                dr.gsel[q] = s;
                break;
            }
            acc += v[j];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
        hist[t] = 0u;
}

// Apply blocks are graph-aligned chunks of GS_CHUNK keys: chunk c of the
// launch belongs to graph q with chunk_off[q] <= c < chunk_off[q + 1].
__device__ __forceinline__ void chunk_range(const DevGraph &g, const DevRun &dr, bool rs, int c, int &q, int &x0,
                                            int &x1)
{
    const int32_t *co = dr.chunk_off + (rs ? g.G + 1 : 0);
    q = graph_of(co, g.G, c);
    const int32_t *off = rs ? g.gv_off : g.ge_off;
    x0 = off[q] + (c - co[q]) * GS_CHUNK;
    x1 = min(off[q + 1], x0 + GS_CHUNK);
}

// Keys equal to the threshold per chunk (only graphs whose ties straddle it).
template <typename RT, bool RS>
__global__ void __launch_bounds__(GS_THREADS) k_gsel_tiecount(DevGraph g, DevRun dr)
{
    using KeyT = decltype(gkey((RT)0));
    __shared__ int s_cnt;
    int q, x0, x1;
    chunk_range(g, dr, RS, blockIdx.x, q, x0, x1);
    if (dr.gs[q].status != ST_RUNNING)
        return;
    const GSelState s = dr.gsel[q];
    if (s.krem == s.eq_total)
        return;   // every tie is taken: no ranking
    if (threadIdx.x == 0)
        s_cnt = 0;
    __syncthreads();
    int c = 0;
    for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x)
        c += key_at<RT, RS>(dr, x) == (KeyT)s.prefix;
    if (c)
        atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0)
        dr.gsel_tie[blockIdx.x] = s_cnt;
}

// Exclusive scan of the tie counts over the chunks of each graph (one block
// per graph, sequential over warps of 32 chunks).
__global__ void __launch_bounds__(32) k_gsel_tiescan(DevGraph g, DevRun dr, bool rs)
{
    const int q = blockIdx.x;
    if (dr.gs[q].status != ST_RUNNING)
        return;
    const GSelState s = dr.gsel[q];
    if (s.krem == s.eq_total)
        return;
    const int32_t *co = dr.chunk_off + (rs ? g.G + 1 : 0);
    const int c0 = co[q], c1 = co[q + 1];
    const int lane = threadIdx.x;
    int carry = 0;
    for (int base = c0; base < c1; base += 32) {
        const int c = base + lane;
        const int v = c < c1 ? dr.gsel_tie[c] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (c < c1)
            dr.gsel_tie[c] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Takes every key above the threshold and the first krem keys equal to it
// (by index). RBP copies the selected candidates into the state buffer; RS
// sets the splash level (0 = root, -1 = not reached yet).
template <typename S, typename RT, bool RS>
__global__ void __launch_bounds__(GS_THREADS) k_gsel_apply(DevGraph g, DevRun dr, RunParams rp)
{
    using KeyT = decltype(gkey((RT)0));
    __shared__ int warp_cnt[GS_THREADS / 32];
    int q, x0, x1;
    chunk_range(g, dr, RS, blockIdx.x, q, x0, x1);
    const GState st = dr.gs[q];
    if (st.status != ST_RUNNING)
        return;
    const GSelState s = dr.gsel[q];
    const KeyT thr = (KeyT)s.prefix;
    const bool rank_ties = s.krem != s.eq_total;
    const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
    const int epm = g.epm;
    S *dst = (S *)dr.msg[0];
    const S *src = (const S *)dr.msg[1];
    int before = rank_ties ? dr.gsel_tie[blockIdx.x] : 0;   // ties in earlier chunks of the graph
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = x0; base < x1; base += blockDim.x) {
        const int x = base + threadIdx.x;
        const bool in = x < x1;
        const KeyT k = in ? key_at<RT, RS>(dr, x) : (KeyT)0;
        bool take = in && k > thr;
        if (rank_ties) {
            const bool eq = in && k == thr;
            const unsigned b = __ballot_sync(0xffffffffu, eq);
            if (lane == 0)
                warp_cnt[warp] = __popc(b);
            __syncthreads();
            int r = before + __popc(b & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w)
                r += warp_cnt[w];
            take = take || (eq && r < s.krem);
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                tot += warp_cnt[w];
            __syncthreads();
            before += tot;
        } else {
            take = take || (in && k == thr);
        }
        if (!in)
            continue;
        if (RS) {
            dr.level[x] = take ? (int8_t)0 : (int8_t)-1;
        } else if (take) {
            for (int j = 0; j < epm; ++j)
                dst[(size_t)x * epm + j] = src[(size_t)x * epm + j];
        }
        if (take && tr)
            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (x >> 5)], 1u << (x & 31));
    }
}

template <typename S, typename RT, bool RS>
static void run_grid_select(const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    using KeyT = decltype(gkey((RT)0));
    using D = Digits<KeyT>;
    const int nb_hist = 152 * 4;
    if (RS)
        k_gsel_vres<RT><<<152 * 4, GS_THREADS, 0, s>>>(g, dr);
    k_gsel_init<<<(g.G + 127) / 128, 128, 0, s>>>(g, dr);
    for (int p = 0; p < D::passes; ++p) {
        k_gsel_hist<RT, RS><<<nb_hist, GS_THREADS, 0, s>>>(g, dr, p);
        k_gsel_digit<RT><<<g.G, 1024, 0, s>>>(g, dr, p);
    }
    const int chunks = RS ? dr.n_chunks_rs : dr.n_chunks_rbp;
    k_gsel_tiecount<RT, RS><<<chunks, GS_THREADS, 0, s>>>(g, dr);
    k_gsel_tiescan<<<g.G, 32, 0, s>>>(g, dr, RS);
    k_gsel_apply<S, RT, RS><<<chunks, GS_THREADS, 0, s>>>(g, dr, rp);
}

int grid_select_launches(int dtype, bool rs)
{
    const int passes = dtype == DT_F64 ? Digits<unsigned long long>::passes : Digits<uint32_t>::passes;
    return (rs ? 1 : 0) + 1 + 2 * passes + 3;
}

int grid_select_chunks(const int32_t *off, int G, int32_t *chunk_off)
{
    chunk_off[0] = 0;
    for (int q = 0; q < G; ++q)
        chunk_off[q + 1] = chunk_off[q] + (off[q + 1] - off[q] + GS_CHUNK - 1) / GS_CHUNK;
    return chunk_off[G];
}

int grid_select_bins() { return GS_BINS; }

void launch_select_rbp_grid(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    switch (dtype) {
    case DT_F64: run_grid_select<double, double, false>(g, dr, rp, s); break;
    case DT_F32: run_grid_select<float, float, false>(g, dr, rp, s); break;
    case DT_BF16: run_grid_select<__nv_bfloat16, float, false>(g, dr, rp, s); break;
    default: run_grid_select<int16_t, float, false>(g, dr, rp, s); break;
    }
}

void launch_select_rs_grid(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    // the message type is unused by the RS apply
    if (dtype == DT_F64)
        run_grid_select<double, double, true>(g, dr, rp, s);
    else
        run_grid_select<float, float, true>(g, dr, rp, s);
}

}  // namespace bpg
