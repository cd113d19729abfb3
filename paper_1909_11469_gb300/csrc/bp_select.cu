// Frontier selection for Residual BP and Residual Splash (Section III-A):
// exact top-k by residual with ties to the smaller id, one CTA per graph.
//
// The paper sorts (key-value radix sort) and takes the prefix; here a CTA runs
// an MSB radix select on the residual's IEEE bits (non-negative floats order as
// unsigned integers): one 256-bin shared-memory histogram per byte narrows the
// k-th largest key, then an ordered pass takes every key above it and the
// lowest-id ties. The selected RBP messages are committed in the same pass.
#include "bp_internal.cuh"
#include "bp_launch.h"

namespace bpg {

constexpr int SEL_THREADS = 1024;

__device__ __forceinline__ uint32_t key_bits(float v) { return __float_as_uint(v); }
__device__ __forceinline__ unsigned long long key_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v);
}

// Finds thr = the k-th largest key (1 <= k <= count) and take_eq = how many keys
// equal to thr belong to the top k. Every thread of the block must call it.
template <typename KeyT, typename KeyFn>
__device__ void block_select_threshold(int count, int k, KeyFn key, KeyT &thr, int &take_eq)
{
    __shared__ unsigned int hist[256];
    __shared__ KeyT s_prefix;
    __shared__ int s_krem;
    KeyT prefix = 0, mask = 0;
    int krem = k;
    for (int pass = 0; pass < (int)sizeof(KeyT); ++pass) {
        const int shift = ((int)sizeof(KeyT) - 1 - pass) * 8;
        for (int t = threadIdx.x; t < 256; t += blockDim.x)
            hist[t] = 0u;
        __syncthreads();
        for (int idx = threadIdx.x; idx < count; idx += blockDim.x) {
            KeyT kv = key(idx);
            if ((kv & mask) == prefix)
                atomicAdd(&hist[(unsigned)((kv >> shift) & (KeyT)255)], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // lane L owns digits 255-8L down to 248-8L (descending order)
            const int lane = threadIdx.x;
            unsigned loc[8];
            unsigned sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                loc[q] = hist[255 - 8 * lane - q];
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
                s_prefix = prefix | ((KeyT)d << shift);
                s_krem = krem - (int)acc;
            }
        }
        __syncthreads();
        prefix = s_prefix;
        krem = s_krem;
        mask |= ((KeyT)255 << shift);
        __syncthreads();
    }
    thr = prefix;
    take_eq = krem;
}

// Ordered pass: calls on_item(idx, take) for every idx < count, take = key above
// thr, or equal to thr and among the first take_eq such ids.
template <typename KeyT, typename KeyFn, typename ItemFn>
__device__ void block_select_apply(int count, KeyT thr, int take_eq, KeyFn key, ItemFn on_item)
{
    __shared__ unsigned int s_warp[32];
    __shared__ int s_taken;
    if (threadIdx.x == 0)
        s_taken = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < count; base += blockDim.x) {
        const int idx = base + threadIdx.x;
        const bool in = idx < count;
        const KeyT kv = in ? key(idx) : (KeyT)0;
        const bool gt = in && kv > thr;
        const bool eq = in && kv == thr;
        const unsigned b = __ballot_sync(0xffffffffu, eq);
        if (lane == 0)
            s_warp[warp] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w)
            before += (int)s_warp[w];
        const int rank = s_taken + before + __popc(b & ((1u << lane) - 1u));
        if (in)
            on_item(idx, gt || (eq && rank < take_eq));
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nw; ++w)
                tot += (int)s_warp[w];
            s_taken += tot;
        }
        __syncthreads();
    }
}

// RBP: select the top k_sel messages of each running graph and commit them.
template <typename S>
__global__ void __launch_bounds__(SEL_THREADS) k_select_rbp(DevGraph g, DevRun dr, RunParams rp)
{
    using RT = typename ResidT<S>::T;
    using KeyT = decltype(key_bits((RT)0));
    const int gg = blockIdx.x;
    const GState st = dr.gs[gg];
    if (st.status != ST_RUNNING)
        return;
    const int e0 = g.ge_off[gg];
    const int cnt = g.ge_off[gg + 1] - e0;
    if (cnt == 0)
        return;
    const RT *R = (const RT *)dr.resid + e0;
    auto key = [&](int idx) -> KeyT { return key_bits(R[idx]); };
    KeyT thr;
    int take_eq;
    block_select_threshold<KeyT>(cnt, st.k_sel, key, thr, take_eq);
    S *dst = (S *)dr.msg[0];
    const S *src = (const S *)dr.msg[1];
    const int epm = g.epm;
    const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
    block_select_apply<KeyT>(cnt, thr, take_eq, key, [&](int idx, bool take) {
        if (!take)
            return;
        const int e = e0 + idx;
        for (int x = 0; x < epm; ++x)
            dst[(size_t)e * epm + x] = src[(size_t)e * epm + x];
        if (tr)
            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (e >> 5)], 1u << (e & 31));
    });
}

// RS: vertex residual = max residual of the incoming messages; select the top
// k_sel vertices as splash roots (level 0), every other vertex gets level -1.
template <typename S>
__global__ void __launch_bounds__(SEL_THREADS) k_select_rs(DevGraph g, DevRun dr, RunParams rp)
{
    using RT = typename ResidT<S>::T;
    using KeyT = decltype(key_bits((RT)0));
    const int gg = blockIdx.x;
    const GState st = dr.gs[gg];
    if (st.status != ST_RUNNING)
        return;
    const int v0 = g.gv_off[gg];
    const int nv = g.gv_off[gg + 1] - v0;
    if (nv == 0)
        return;
    const RT *R = (const RT *)dr.resid;
    RT *VR = (RT *)dr.vres + v0;
    for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
        const int v = v0 + idx;
        RT m = 0;
        for (int f = g.row_ptr[v]; f < g.row_ptr[v + 1]; ++f) {
            RT r = R[g.rev[f]];
            m = r > m ? r : m;
        }
        VR[idx] = m;
    }
    __syncthreads();
    auto key = [&](int idx) -> KeyT { return key_bits(VR[idx]); };
    KeyT thr;
    int take_eq;
    block_select_threshold<KeyT>(nv, st.k_sel, key, thr, take_eq);
    const bool tr = rp.record_trace && st.rounds <= rp.trace_capacity;
    block_select_apply<KeyT>(nv, thr, take_eq, key, [&](int idx, bool take) {
        const int v = v0 + idx;
        dr.level[v] = take ? (int8_t)0 : (int8_t)-1;
        if (take && tr)
            atomicOr(&dr.trace[(size_t)(st.rounds - 1) * rp.trace_words + (v >> 5)], 1u << (v & 31));
    });
}

void launch_select_rbp(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    switch (dtype) {
    case DT_F64: k_select_rbp<double><<<g.G, SEL_THREADS, 0, s>>>(g, dr, rp); break;
    case DT_F32: k_select_rbp<float><<<g.G, SEL_THREADS, 0, s>>>(g, dr, rp); break;
    case DT_BF16: k_select_rbp<__nv_bfloat16><<<g.G, SEL_THREADS, 0, s>>>(g, dr, rp); break;
    default: k_select_rbp<int16_t><<<g.G, SEL_THREADS, 0, s>>>(g, dr, rp); break;
    }
}

void launch_select_rs(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s)
{
    // selection reads residuals only: FP64 runs keep double residuals, the others float
    if (dtype == DT_F64)
        k_select_rs<double><<<g.G, SEL_THREADS, 0, s>>>(g, dr, rp);
    else
        k_select_rs<float><<<g.G, SEL_THREADS, 0, s>>>(g, dr, rp);
}

}  // namespace bpg
