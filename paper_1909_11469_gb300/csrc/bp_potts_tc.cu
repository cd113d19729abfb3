// Shared-table (Potts) message update on the 5th-generation tensor cores.
//
// With one k x k table Theta shared by every edge, Eq. 2 for a directed edge e
// is a row-vector product: with a_e(x) = exp(cav_e(x) - max cav_e) and
// Psi = exp(Theta), the new message is c_e(y) = sum_x a_e(x) Psi(x, y). A tile of
// 128 edges is the GEMM D[128 x 32] = A[128 x 32] * Psi[32 x 32]: A in BF16 in
// shared memory (no-swizzle K-major core matrices), Psi resident in shared
// memory, D accumulated in FP32 in tensor memory by tcgen05.mma issued from one
// thread, read back row-per-thread with tcgen05.ld. The split mode adds
// A_lo * Psi_hi + A_hi * Psi_lo (BF16 residuals of A and Psi) for close to FP32
// accuracy. States are padded to 32 (k <= 32).
//
// A CTA is one warpgroup (128 threads) and loops over tiles of consecutive
// vertices whose out-edges number at most 128 (tile bounds precomputed on the
// host). Per tile:
//   1. vertex fields S_v(x) = theta_v(x) + sum of incoming logs (lane = state),
//      incoming rows kept in shared memory
//   2. thread = edge: cavity, max, a(x) -> A operand (BF16, hi and lo parts)
//   3. one thread issues the MMAs and commits them to an mbarrier
//   4. thread = edge: D row from TMEM, log + max, normalisation, residual,
//      stores (new message, residual), convergence reduction
// Every mbarrier wait is bounded; on expiry the CTA records an error, waits
// (bounded) for its MMAs, frees its tensor memory and returns.
#include "bp_internal.cuh"
#include "bp_launch.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace bpg {

constexpr int TC_ROWS = 128;    // edges per tile (MMA M)
constexpr int TC_K = 32;        // padded states (MMA N, and K in two steps of 16)
constexpr int TC_VMAX = 32;     // vertices per tile
constexpr int TC_THREADS = 128;
constexpr int TC_TMEM_COLS = 32;
constexpr long long TC_WAIT_LIMIT = 1ll << 22;

// Byte offset of element (row, k) in a no-swizzle K-major BF16 operand of 32
// columns: core matrices of 8 rows x 16 bytes; along K they are 128 B apart
// (leading byte offset), along rows 512 B apart (stride byte offset).
__device__ __forceinline__ int core_offset(int row, int k)
{
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

struct TcShared {
    unsigned char a_hi[TC_ROWS * TC_K * 2];
    unsigned char a_lo[TC_ROWS * TC_K * 2];
    unsigned char b_hi[TC_K * TC_K * 2];
    unsigned char b_lo[TC_K * TC_K * 2];
    float stash[TC_ROWS][TC_K + 1];   // incoming message of each edge (log), padded row
    float S[TC_VMAX][TC_K + 1];       // vertex fields
    int src_local[TC_ROWS];
    int rev_t[TC_ROWS];               // rev of the tile's edges
    int cur_of[TC_VMAX];              // message buffer of the vertex's graph, -1 inactive
    unsigned long long mbar;
    unsigned int tmem_base;
    int err;
    double w_max[4];
    unsigned int w_cnt[4];
    float psi_f[TC_K][TC_K];          // CUDA-core form of Psi (x, y)
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4, leading / stride byte offsets
// >> 4, descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long make_desc(const void *p, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((smem_u32(p) >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 32, M = 128.
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TC_K >> 3) << 17) |
                              ((unsigned)(TC_ROWS >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, unsigned parity)
{
    const unsigned a = smem_u32(mbar);
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
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

// TC = true: contraction on the tensor cores; TC = false: the same tile
// pipeline with the contraction on the CUDA cores (FP32 FMAs against Psi in
// shared memory), as the CUDA-core twin.
template <typename S, int MODE, bool TC>
__global__ void __launch_bounds__(TC_THREADS) k_potts_tc(DevGraph g, DevRun dr, RunParams rp, const int *tile_v,
                                                         int n_tiles, int split, int *err_flag)
{
    using RT = typename ResidT<S>::T;
    extern __shared__ unsigned char tc_raw[];
    TcShared &sh = *reinterpret_cast<TcShared *>(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = g.k;

    // Psi = exp(Theta - max Theta) as B operands (hi and lo BF16 parts), padded.
    for (int idx = tid; idx < TC_K * TC_K; idx += TC_THREADS) {
        const int y = idx / TC_K, x = idx % TC_K;      // B row n = y, column k = x
        const float psi = (x < k && y < k) ? g.psi_shared[x * k + y] : 0.0f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(psi);
        const __nv_bfloat16 lo = __float2bfloat16_rn(psi - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16 *>(sh.b_hi + core_offset(y, x)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(sh.b_lo + core_offset(y, x)) = lo;
        sh.psi_f[x][y] = psi;
    }
    if (tid == 0) {
        sh.err = 0;
        if (TC) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.mbar)));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
    }
    if (TC && warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = TC ? sh.tmem_base : 0u;
    const float floor_log = -80.0f;
    unsigned phase = 0;
    bool failed = false;

    for (int tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        const int va = tile_v[tile], vb = tile_v[tile + 1];
        const int nvt = vb - va;
        const int e0 = g.row_ptr[va];
        const int ne = g.row_ptr[vb] - e0;
        // 0. vertex pass: graph state and source vertex of every edge
        if (tid < nvt) {
            const int v = va + tid;
            const int gg = g.gid[v];
            sh.cur_of[tid] = dr.gs[gg].status == ST_RUNNING ? dr.gs[gg].cur : -1;
            for (int e = g.row_ptr[v]; e < g.row_ptr[v + 1]; ++e)
                sh.src_local[e - e0] = tid;
        }
        if (tid < ne)
            sh.rev_t[tid] = g.rev[e0 + tid];
        __syncthreads();
        // 1. incoming rows of the tile's edges: independent 16-byte loads (8 per
        //    thread in flight for k = 32), then vertex fields from shared memory
        if (k == TC_K && sizeof(S) == 4) {
            float4 v4[TC_ROWS * (TC_K / 4) / TC_THREADS];
#pragma unroll
            for (int j = 0; j < TC_ROWS * (TC_K / 4) / TC_THREADS; ++j) {
                const int idx = tid + j * TC_THREADS;
                const int er = idx >> 3, ch = idx & 7;
                v4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (er < ne) {
                    const int c = sh.cur_of[sh.src_local[er]];
                    if (c >= 0)
                        v4[j] = *reinterpret_cast<const float4 *>((const float *)msg_buf(dr, c) +
                                                                  (size_t)sh.rev_t[er] * TC_K + 4 * ch);
                }
            }
#pragma unroll
            for (int j = 0; j < TC_ROWS * (TC_K / 4) / TC_THREADS; ++j) {
                const int idx = tid + j * TC_THREADS;
                const int er = idx >> 3, ch = idx & 7;
                if (er < ne) {
                    sh.stash[er][4 * ch + 0] = v4[j].x;
                    sh.stash[er][4 * ch + 1] = v4[j].y;
                    sh.stash[er][4 * ch + 2] = v4[j].z;
                    sh.stash[er][4 * ch + 3] = v4[j].w;
                }
            }
        } else {
            for (int idx = tid; idx < ne * TC_K; idx += TC_THREADS) {
                const int er = idx / TC_K, x = idx % TC_K;
                const int c = sh.cur_of[sh.src_local[er]];
                float in = 0.0f;
                if (c >= 0 && x < k)
                    in = Store<S>::ld((const S *)msg_buf(dr, c) + (size_t)sh.rev_t[er] * k + x, g.qscale);
                sh.stash[er][x] = in;
            }
        }
        __syncthreads();
        for (int vl = warp; vl < nvt; vl += 4) {
            const int v = va + vl;
            float sv = (lane < k) ? g.unary[(size_t)v * k + lane] : 0.0f;
            for (int e = g.row_ptr[v] - e0; e < g.row_ptr[v + 1] - e0; ++e)
                sv += sh.stash[e][lane];
            sh.S[vl][lane] = sv;
        }
        __syncthreads();
        // 2. A operand: thread = edge row
        const int row = tid;
        const bool has_row = row < ne;
        const int src = has_row ? sh.src_local[row] : 0;
        const int c_row = has_row ? sh.cur_of[src] : -1;
        float mx = -1e30f;
        if (has_row)
            for (int x = 0; x < k; ++x)
                mx = fmaxf(mx, sh.S[src][x] - sh.stash[row][x]);
        float d[TC_K];
        if (!TC) {
            float a[TC_K];
#pragma unroll
            for (int x = 0; x < TC_K; ++x)
                a[x] = (has_row && x < k) ? __expf(sh.S[src][x] - sh.stash[row][x] - mx) : 0.0f;
#pragma unroll
            for (int y = 0; y < TC_K; ++y) {
                float acc = 0.0f;
#pragma unroll
                for (int x = 0; x < TC_K; ++x)
                    acc = fmaf(a[x], sh.psi_f[x][y], acc);
                d[y] = acc;
            }
        } else {
    #pragma unroll
            for (int xb = 0; xb < TC_K; xb += 8) {
                unsigned hw[4], lw[4];
    #pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    unsigned hb[2], lb[2];
    #pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const int x = xb + j + t;
                        float a = 0.0f;
                        if (has_row && x < k)
                            a = __expf(sh.S[src][x] - sh.stash[row][x] - mx);
                        const __nv_bfloat16 h = __float2bfloat16_rn(a);
                        const __nv_bfloat16 l = __float2bfloat16_rn(a - __bfloat162float(h));
                        hb[t] = __bfloat16_as_ushort(h);
                        lb[t] = __bfloat16_as_ushort(l);
                    }
                    hw[j / 2] = hb[0] | (hb[1] << 16);   // element x at the lower address
                    lw[j / 2] = lb[0] | (lb[1] << 16);
                }
                *reinterpret_cast<uint4 *>(sh.a_hi + core_offset(row, xb)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(sh.a_lo + core_offset(row, xb)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            // 3. MMAs from one thread: D = A_hi Psi_hi (+ A_lo Psi_hi + A_hi Psi_lo)
            if (tid == 0) {
    #pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    mma_bf16(tmem, make_desc(sh.a_hi + ks * 256, 128, 512), make_desc(sh.b_hi + ks * 256, 128, 512),
                             ks > 0);
                }
                if (split) {
    #pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        mma_bf16(tmem, make_desc(sh.a_lo + ks * 256, 128, 512),
                                 make_desc(sh.b_hi + ks * 256, 128, 512), 1);
                        mma_bf16(tmem, make_desc(sh.a_hi + ks * 256, 128, 512),
                                 make_desc(sh.b_lo + ks * 256, 128, 512), 1);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&sh.mbar)));
            }
            if (!mbar_wait(&sh.mbar, phase)) {
                failed = true;
                if (tid == 0)
                    sh.err = 1;
            }
            phase ^= 1u;
            __syncthreads();
            if (sh.err) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // 4. epilogue: D row of this thread from TMEM (warp w reads lanes 32w..32w+31)
            {
                unsigned r[TC_K];
                const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                             "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
                             "%28, %29, %30, %31}, [%32];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                               "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                               "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                               "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    #pragma unroll
                for (int j = 0; j < TC_K; ++j)
                    d[j] = __uint_as_float(r[j]);
            }
        }
        float maxr = 0.0f;
        unsigned cnt = 0;
        const bool uniform_tile = g.gid[va] == g.gid[vb - 1];
        if (has_row && c_row >= 0) {
            const int e = e0 + row;
            float z = 0.0f;
#pragma unroll
            for (int y = 0; y < TC_K; ++y)
                if (y < k)
                    z += d[y];
            const S *old = (const S *)msg_buf(dr, c_row) + (size_t)e * k;
            S *out = (S *)msg_buf(dr, MODE == MODE_LBP ? (c_row ^ 1) : 1) + (size_t)e * k;
            float r = 0.0f;
            if (k == TC_K && sizeof(S) == 4) {
                float4 o4[TC_K / 4];
#pragma unroll
                for (int j = 0; j < TC_K / 4; ++j)
                    o4[j] = reinterpret_cast<const float4 *>(old)[j];
                const float iz = __fdividef(1.0f, z);
#pragma unroll
                for (int j = 0; j < TC_K / 4; ++j) {
                    float l[4];
                    const float ov[4] = {o4[j].x, o4[j].y, o4[j].z, o4[j].w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float pn = d[4 * j + t] * iz;
                        l[t] = fmaxf(__logf(pn), floor_log);
                        r = fmaxf(r, fabsf(__expf(l[t]) - __expf(ov[t])));
                    }
                    reinterpret_cast<float4 *>(out)[j] = make_float4(l[0], l[1], l[2], l[3]);
                }
            } else {
#pragma unroll
                for (int y = 0; y < TC_K; ++y) {
                    if (y < k) {
                        float lnew = __logf(__fdividef(d[y], z));
                        lnew = lnew > floor_log ? lnew : floor_log;
                        const float pn = __expf(Store<S>::quant(lnew, g.qscale));
                        const float po = __expf(Store<S>::ld(old + y, g.qscale));
                        r = fmaxf(r, fabsf(pn - po));
                        Store<S>::st(out + y, lnew, g.qscale);
                    }
                }
            }
            if (MODE == MODE_CAND)
                ((RT *)dr.resid)[e] = (RT)r;
            maxr = r;
            cnt = (r >= eps_in(rp, 0.0f)) ? 1u : 0u;
            if (!uniform_tile) {
                // tile spanning graphs: account the message to its own graph
                const int gg = g.gid[va + src];
                const int slot = blockIdx.x & (NSUB - 1);
                if (r > 0.0f)
                    atomicMax(&dr.red_max[(size_t)gg * NSUB + slot],
                              (unsigned long long)__double_as_longlong((double)r));
                if (cnt)
                    atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], 1u);
            }
        }
        if (uniform_tile) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                maxr = fmaxf(maxr, __shfl_xor_sync(0xffffffffu, maxr, o));
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            }
            if (lane == 0) {
                sh.w_max[warp] = maxr;
                sh.w_cnt[warp] = cnt;
            }
            __syncthreads();
            if (tid == 0) {
                double m = 0.0;
                unsigned c = 0;
                for (int w = 0; w < 4; ++w) {
                    m = fmax(m, sh.w_max[w]);
                    c += sh.w_cnt[w];
                }
                const int gg = g.gid[va];
                const int slot = blockIdx.x & (NSUB - 1);
                if (m > 0.0)
                    atomicMax(&dr.red_max[(size_t)gg * NSUB + slot], (unsigned long long)__double_as_longlong(m));
                if (c)
                    atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], c);
            }
        }
        // TMEM is overwritten by the next tile's MMAs only after every thread read it
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (failed) {
        if (tid == 0)
            atomicExch(err_flag, 1);
        // the MMAs of the failed tile may still be in flight: wait (bounded) once more
        mbar_wait(&sh.mbar, phase ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (TC && warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ---------------------------------------------------------------------------
// Pipelined form for FP32 messages with k = 32 (every state a full 128-byte
// row): the incoming rows of the CTA's next tile are copied into a second
// shared-memory stage with cp.async (16-byte chunks, zero-filled for inactive
// rows) while the current tile runs its vertex fields, contraction and
// epilogue, so the gather latency overlaps the arithmetic. The arithmetic is
// that of k_potts_tc (same operations in the same order). Used for the
// CUDA-core contraction; with the tensor cores the smaller single-stage CTA
// (4 per SM instead of 3) measured faster.
constexpr int TP_STRIDE = 36;   // floats per staged row: 16-byte aligned, conflict-free float4 reads

struct TcPipeShared {
    unsigned char a_hi[TC_ROWS * TC_K * 2];
    unsigned char a_lo[TC_ROWS * TC_K * 2];
    unsigned char b_hi[TC_K * TC_K * 2];
    unsigned char b_lo[TC_K * TC_K * 2];
    float stash[2][TC_ROWS][TP_STRIDE];   // incoming message of each edge (log), two stages
    float S[TC_VMAX][TP_STRIDE];          // vertex fields
    int src_local[2][TC_ROWS];
    int rev_t[2][TC_ROWS];
    int cur_of[2][TC_VMAX];
    unsigned long long mbar;
    unsigned int tmem_base;
    int err;
    double w_max[4];
    unsigned int w_cnt[4];
    float psi_f[TC_K][TC_K];
};

// Tile metadata into stage b: source vertex of every edge, rev of every edge,
// message buffer of every vertex's graph (-1: graph not running).
__device__ __forceinline__ void tp_meta(const DevGraph &g, const DevRun &dr, const int *tile_v, int tile,
                                        TcPipeShared &sh, int b, int tid)
{
    const int va = tile_v[tile], vb = tile_v[tile + 1];
    const int nvt = vb - va;
    const int e0 = g.row_ptr[va];
    const int ne = g.row_ptr[vb] - e0;
    if (tid < nvt) {
        const int v = va + tid;
        const int gg = g.gid[v];
        sh.cur_of[b][tid] = dr.gs[gg].status == ST_RUNNING ? dr.gs[gg].cur : -1;
        for (int e = g.row_ptr[v]; e < g.row_ptr[v + 1]; ++e)
            sh.src_local[b][e - e0] = tid;
    }
    if (tid < ne)
        sh.rev_t[b][tid] = g.rev[e0 + tid];
}

// Asynchronous copy of the tile's incoming rows into stage b (8 chunks of
// 16 bytes per row, 8 per thread), committed as one group.
__device__ __forceinline__ void tp_gather(const DevGraph &g, const DevRun &dr, const int *tile_v, int tile,
                                          TcPipeShared &sh, int b, int tid)
{
    const int va = tile_v[tile], vb = tile_v[tile + 1];
    const int ne = g.row_ptr[vb] - g.row_ptr[va];
    const float *base = (const float *)dr.msg[0];
#pragma unroll
    for (int j = 0; j < TC_ROWS * (TC_K / 4) / TC_THREADS; ++j) {
        const int idx = tid + j * TC_THREADS;
        const int er = idx >> 3, ch = idx & 7;
        const float *src = base;
        unsigned bytes = 0;
        if (er < ne) {
            const int c = sh.cur_of[b][sh.src_local[b][er]];
            if (c >= 0) {
                src = (const float *)msg_buf(dr, c) + (size_t)sh.rev_t[b][er] * TC_K + 4 * ch;
                bytes = 16;
            }
        }
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(&sh.stash[b][er][4 * ch])),
                     "l"(src), "r"(bytes)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int MODE, bool TC>
__global__ void __launch_bounds__(TC_THREADS) k_potts_tc_pipe(DevGraph g, DevRun dr, RunParams rp,
                                                              const int *tile_v, int n_tiles, int split,
                                                              int *err_flag)
{
    using S = float;
    extern __shared__ unsigned char tc_raw[];
    TcPipeShared &sh = *reinterpret_cast<TcPipeShared *>(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int idx = tid; idx < TC_K * TC_K; idx += TC_THREADS) {
        const int y = idx / TC_K, x = idx % TC_K;
        const float psi = g.psi_shared[x * TC_K + y];
        const __nv_bfloat16 hi = __float2bfloat16_rn(psi);
        const __nv_bfloat16 lo = __float2bfloat16_rn(psi - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16 *>(sh.b_hi + core_offset(y, x)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(sh.b_lo + core_offset(y, x)) = lo;
        sh.psi_f[x][y] = psi;
    }
    if (tid == 0) {
        sh.err = 0;
        if (TC) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sh.mbar)));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
    }
    if (TC && warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = TC ? sh.tmem_base : 0u;
    const float floor_log = -80.0f;
    unsigned phase = 0;
    bool failed = false;

    // prologue: stage 0 holds the first tile
    int tile = blockIdx.x;
    if (tile < n_tiles) {
        tp_meta(g, dr, tile_v, tile, sh, 0, tid);
        __syncthreads();
        tp_gather(g, dr, tile_v, tile, sh, 0, tid);
    }
    for (int it = 0; tile < n_tiles && !failed; ++it, tile += gridDim.x) {
        const int b = it & 1;
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();   // stage b complete for every thread
        const int next = tile + gridDim.x;
        if (next < n_tiles) {
            tp_meta(g, dr, tile_v, next, sh, b ^ 1, tid);
            __syncthreads();
            tp_gather(g, dr, tile_v, next, sh, b ^ 1, tid);   // lands while this tile computes
        }
        const int va = tile_v[tile], vb = tile_v[tile + 1];
        const int nvt = vb - va;
        const int e0 = g.row_ptr[va];
        const int ne = g.row_ptr[vb] - e0;
        // 1. vertex fields from the staged rows (lane = state)
        for (int vl = warp; vl < nvt; vl += 4) {
            const int v = va + vl;
            float sv = g.unary[(size_t)v * TC_K + lane];
            for (int e = g.row_ptr[v] - e0; e < g.row_ptr[v + 1] - e0; ++e)
                sv += sh.stash[b][e][lane];
            sh.S[vl][lane] = sv;
        }
        __syncthreads();
        // 2. A operand: thread = edge row
        const int row = tid;
        const bool has_row = row < ne;
        const int src = has_row ? sh.src_local[b][row] : 0;
        const int c_row = has_row ? sh.cur_of[b][src] : -1;
        float mx = -1e30f;
        if (has_row) {
#pragma unroll
            for (int x = 0; x < TC_K; x += 4) {
                const float4 sv = *reinterpret_cast<const float4 *>(&sh.S[src][x]);
                const float4 iv = *reinterpret_cast<const float4 *>(&sh.stash[b][row][x]);
                mx = fmaxf(mx, sv.x - iv.x);
                mx = fmaxf(mx, sv.y - iv.y);
                mx = fmaxf(mx, sv.z - iv.z);
                mx = fmaxf(mx, sv.w - iv.w);
            }
        }
        float d[TC_K];
        if (!TC) {
            float a[TC_K];
#pragma unroll
            for (int x = 0; x < TC_K; ++x)
                a[x] = has_row ? __expf(sh.S[src][x] - sh.stash[b][row][x] - mx) : 0.0f;
#pragma unroll
            for (int y = 0; y < TC_K; ++y) {
                float acc = 0.0f;
#pragma unroll
                for (int x = 0; x < TC_K; ++x)
                    acc = fmaf(a[x], sh.psi_f[x][y], acc);
                d[y] = acc;
            }
        } else {
#pragma unroll
            for (int xb = 0; xb < TC_K; xb += 8) {
                unsigned hw[4], lw[4];
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    unsigned hb[2], lb[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const int x = xb + j + t;
                        const float a = has_row ? __expf(sh.S[src][x] - sh.stash[b][row][x] - mx) : 0.0f;
                        const __nv_bfloat16 h = __float2bfloat16_rn(a);
                        const __nv_bfloat16 l = __float2bfloat16_rn(a - __bfloat162float(h));
                        hb[t] = __bfloat16_as_ushort(h);
                        lb[t] = __bfloat16_as_ushort(l);
                    }
                    hw[j / 2] = hb[0] | (hb[1] << 16);
                    lw[j / 2] = lb[0] | (lb[1] << 16);
                }
                *reinterpret_cast<uint4 *>(sh.a_hi + core_offset(row, xb)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4 *>(sh.a_lo + core_offset(row, xb)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            // 3. MMAs from one thread
            if (tid == 0) {
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    mma_bf16(tmem, make_desc(sh.a_hi + ks * 256, 128, 512), make_desc(sh.b_hi + ks * 256, 128, 512),
                             ks > 0);
                if (split) {
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        mma_bf16(tmem, make_desc(sh.a_lo + ks * 256, 128, 512),
                                 make_desc(sh.b_hi + ks * 256, 128, 512), 1);
                        mma_bf16(tmem, make_desc(sh.a_hi + ks * 256, 128, 512),
                                 make_desc(sh.b_lo + ks * 256, 128, 512), 1);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&sh.mbar)));
            }
            if (!mbar_wait(&sh.mbar, phase)) {
                failed = true;
                if (tid == 0)
                    sh.err = 1;
            }
            phase ^= 1u;
            __syncthreads();
            if (sh.err) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // 4. epilogue: D row of this thread from TMEM
            {
                unsigned r[TC_K];
                const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                             "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
                             "%28, %29, %30, %31}, [%32];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                               "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                               "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                               "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < TC_K; ++j)
                    d[j] = __uint_as_float(r[j]);
            }
        }
        float maxr = 0.0f;
        unsigned cnt = 0;
        const bool uniform_tile = g.gid[va] == g.gid[vb - 1];
        if (has_row && c_row >= 0) {
            const int e = e0 + row;
            float z = 0.0f;
#pragma unroll
            for (int y = 0; y < TC_K; ++y)
                z += d[y];
            const S *old = (const S *)msg_buf(dr, c_row) + (size_t)e * TC_K;
            S *out = (S *)msg_buf(dr, MODE == MODE_LBP ? (c_row ^ 1) : 1) + (size_t)e * TC_K;
            float r = 0.0f;
            float4 o4[TC_K / 4];
#pragma unroll
            for (int j = 0; j < TC_K / 4; ++j)
                o4[j] = reinterpret_cast<const float4 *>(old)[j];
            const float iz = __fdividef(1.0f, z);
#pragma unroll
            for (int j = 0; j < TC_K / 4; ++j) {
                float l[4];
                const float ov[4] = {o4[j].x, o4[j].y, o4[j].z, o4[j].w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const float pn = d[4 * j + t] * iz;
                    l[t] = fmaxf(__logf(pn), floor_log);
                    r = fmaxf(r, fabsf(__expf(l[t]) - __expf(ov[t])));
                }
                reinterpret_cast<float4 *>(out)[j] = make_float4(l[0], l[1], l[2], l[3]);
            }
            if (MODE == MODE_CAND)
                ((float *)dr.resid)[e] = r;
            maxr = r;
            cnt = (r >= eps_in(rp, 0.0f)) ? 1u : 0u;
            if (!uniform_tile) {
                const int gg = g.gid[va + src];
                const int slot = blockIdx.x & (NSUB - 1);
                if (r > 0.0f)
                    atomicMax(&dr.red_max[(size_t)gg * NSUB + slot],
                              (unsigned long long)__double_as_longlong((double)r));
                if (cnt)
                    atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], 1u);
            }
        }
        if (uniform_tile) {
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                maxr = fmaxf(maxr, __shfl_xor_sync(0xffffffffu, maxr, o));
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            }
            if (lane == 0) {
                sh.w_max[warp] = maxr;
                sh.w_cnt[warp] = cnt;
            }
            __syncthreads();
            if (tid == 0) {
                double m = 0.0;
                unsigned c = 0;
                for (int w = 0; w < 4; ++w) {
                    m = fmax(m, sh.w_max[w]);
                    c += sh.w_cnt[w];
                }
                const int gg = g.gid[va];
                const int slot = blockIdx.x & (NSUB - 1);
                if (m > 0.0)
                    atomicMax(&dr.red_max[(size_t)gg * NSUB + slot], (unsigned long long)__double_as_longlong(m));
                if (c)
                    atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], c);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    // copies still in flight (a failed tile leaves early) land before the CTA exits
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (failed) {
        if (tid == 0)
            atomicExch(err_flag, 1);
        mbar_wait(&sh.mbar, phase ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (TC && warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ---------------------------------------------------------------------------
// Warp-specialised form for k = 32 (FP32 or BF16 messages): one producer warp
// and one consumer warpgroup per CTA.
//
// The producer warp stages whole tiles ahead of the consumers in a ring of
// WS_STAGES shared-memory stages with the tensor-memory-access engine: the
// incoming rows m_{rev(e)} of the tile's 128 edges as 32 four-row gathers
// (cp.async.bulk.tensor .tile::gather4 on a one-row box of the message
// buffer, rows unswizzled) and the unary rows of its (contiguous) vertices as
// one 32-row tile (128-byte swizzle), completion counted in bytes on the
// stage's "full" mbarrier. The tile's static record (vertex and edge range,
// local rows of every vertex, source vertex and rev of every row) is read one
// tile ahead; the producer adds the message buffer of every vertex's graph
// (-1: the graph is not running, its outputs are skipped). Once the consumers
// have built the A operand from the incoming rows, one consumer thread loads
// the old rows m_e of the tile's (contiguous) edges as one 128-row tile into
// the same region, swizzled (128-byte; 64-byte for BF16 messages) so that a
// thread reading its own row hits every bank once; it is in flight while the
// MMAs run, and sharing the region keeps a stage small. (Earlier producers
// measured slower: one 1-D bulk copy per row, ~290 copy requests a tile, and
// 16-byte cp.async copies, whose issue from one warp took ~11k cycles a tile.)
//
// The four consumer warps run the tile pipeline of k_potts_tc on the staged
// rows -- vertex fields (warp = eight vertices side by side, lane = state), A
// operand (thread = edge row, BF16 hi / lo parts), tcgen05.mma from one thread
// into tensor memory, epilogue (thread = row: normalisation, log, residual
// against the staged old row, stores) -- and release the stage with one
// arrival per warp on its "empty" mbarrier. Consumer warp w reads
// tensor-memory lanes 32 (w mod 4) .. + 31, so its rows are those lanes. The
// arithmetic is k_potts_tc's, in the same order. Every wait is bounded; a
// consumer that gives up makes all four warps leave together at the next
// consumer barrier (the barrier ORs their flags), wait (bounded) for their
// last MMA and copies, and free the tensor memory.
constexpr int WS_STAGES = 2;
constexpr int WS_CONS = 4;                       // consumer warps: tensor-memory lanes 0..127
constexpr int WS_THREADS = 32 * (WS_CONS + 1);   // + the producer warp (warp 0)

// Tile metadata of a stage, written by the producer: the tile's static record,
// the message buffer of every vertex's graph (-1: the graph is not running)
// and the buffer every running graph of the tile reads (all the same).
struct WsMeta {
    TcTileRec rec;
    int cur_of[TC_VMAX];
    int buf;
    int pad_[3];
};

// Tensor maps of a launch: the message buffers as [M rows x 32 states] with a
// one-row box (gathers, no swizzle) and a 128-row box (old rows, swizzled),
// the unary log-potentials as [n rows x 32 states] with a 32-row box
// (swizzled).
struct alignas(128) WsMaps {
    CUtensorMap in[2];
    CUtensorMap old[2];
    CUtensorMap un;
};

template <typename S> struct WsLayout {
    static constexpr int ROWB = TC_K * (int)sizeof(S);     // one stored message
    // ROWS holds the incoming rows (unswizzled) until the A operand is built,
    // then the old rows of the tile's edges (swizzled)
    static constexpr int ROWS = 0;                          // [TC_ROWS] rows
    static constexpr int UN = ROWS + TC_ROWS * ROWB;        // [TC_VMAX] unary rows (float, 128-byte swizzle)
    static constexpr int META = UN + TC_VMAX * TC_K * 4;
    static constexpr int STAGE = (META + (int)sizeof(WsMeta) + 1023) / 1024 * 1024;   // swizzle atoms stay aligned
    static constexpr int TX = TC_ROWS * ROWB + TC_VMAX * TC_K * 4;                    // bytes the producer brings
    static constexpr int TX_OLD = TC_ROWS * ROWB;                                     // bytes of the old rows
    static constexpr int A_HI = WS_STAGES * STAGE;
    static constexpr int A_LO = A_HI + TC_ROWS * TC_K * 2;
    static constexpr int B_HI = A_LO + TC_ROWS * TC_K * 2;
    static constexpr int B_LO = B_HI + TC_K * TC_K * 2;
    static constexpr int SF = B_LO + TC_K * TC_K * 2;       // vertex fields [TC_VMAX][TP_STRIDE]
    static constexpr int BAR = SF + TC_VMAX * TP_STRIDE * 4; // full[2], empty[2], mma, old, tmem base
    static constexpr int TOTAL = BAR + 64;
};

// Byte offset of 16-byte chunk c of row r in a swizzled region: the chunk
// index is XORed with the row's position in the 1024-byte swizzle atom
// (128-byte rows: bits 7..9 of the offset; 64-byte rows: bits 7..8).
template <int ROWB> __device__ __forceinline__ int swz(int r, int c)
{
    if constexpr (ROWB == 128)
        return r * 128 + ((c ^ (r & 7)) << 4);
    else
        return r * 64 + ((c ^ ((r >> 1) & 3)) << 4);
}

__device__ __forceinline__ void ws_mbar_init(unsigned a, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void ws_arrive(unsigned a)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void ws_expect_tx(unsigned a, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool ws_wait(unsigned a, unsigned parity)
{
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
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
// Four rows (y0..y3) of a 2-D tensor with a one-row box into consecutive box
// rows at dst; completion on mbar.
__device__ __forceinline__ void ws_gather4(unsigned dst, const CUtensorMap *map, int y0, int y1, int y2, int y3,
                                           unsigned mbar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(mbar)
                 : "memory");
}
// One box of a 2-D tensor starting at row y (column 0); completion on mbar.
__device__ __forceinline__ void ws_tile2d(unsigned dst, const CUtensorMap *map, int y, unsigned mbar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(y), "r"(mbar)
                 : "memory");
}
// Barrier of the four consumer warps (the producer does not take part).
__device__ __forceinline__ void ws_cons_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// The same barrier, returning whether any consumer thread passed fail = true
// (the OR is taken by the barrier itself, so every thread gets the same answer).
__device__ __forceinline__ bool ws_cons_sync_or(bool fail)
{
    unsigned r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 128, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}\n"
                 : "=r"(r)
                 : "r"((unsigned)fail)
                 : "memory");
    return r != 0;
}

// (max residual, count) of this warp's rows of graph gg into a reduction sub-slot.
__device__ __forceinline__ void ws_flush(const DevRun &dr, int gg, float maxr, unsigned cnt, int slot)
{
    const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(maxr));
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && gg >= 0) {
        if (mb)
            atomicMax(&dr.red_max[(size_t)gg * NSUB + slot],
                      (unsigned long long)__double_as_longlong((double)__uint_as_float(mb)));
        if (cnt)
            atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], cnt);
    }
}

// 16-byte chunk c of row r of an unswizzled row region.
template <typename S> __device__ __forceinline__ uint4 ws_chunk(const unsigned char *region, int r, int c)
{
    return reinterpret_cast<const uint4 *>(region + r * TC_K * (int)sizeof(S))[c];
}
// The values of a 16-byte chunk of messages as floats (4 FP32 or 8 BF16 words).
template <typename S> __device__ __forceinline__ void ws_unpack(const uint4 w, float *v, float qs)
{
    if constexpr (sizeof(S) == 4) {
        v[0] = __uint_as_float(w.x);
        v[1] = __uint_as_float(w.y);
        v[2] = __uint_as_float(w.z);
        v[3] = __uint_as_float(w.w);
    } else {
        const unsigned wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int t = 0; t < 8; ++t)
            v[t] = Store<S>::val(__ushort_as_bfloat16((unsigned short)(wv[t >> 1] >> (16 * (t & 1)))), qs);
    }
}

template <typename S, int MODE>
__global__ void __launch_bounds__(WS_THREADS) k_potts_ws(DevGraph g, DevRun dr, RunParams rp,
                                                         const TcTileRec *tile_rec, int n_tiles, int split,
                                                         int *err_flag, const __grid_constant__ WsMaps maps)
{
    using L = WsLayout<S>;
    extern __shared__ unsigned char ws_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)ws_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm + L::BAR);
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(sm + L::BAR + 8 * (2 * WS_STAGES + 2));
    const unsigned full0 = smem_u32(bars), empty0 = smem_u32(bars + WS_STAGES);
    const unsigned mma_bar = smem_u32(bars + 2 * WS_STAGES), old_bar = smem_u32(bars + 2 * WS_STAGES + 1);
    const float qs = g.qscale;

    // Psi = exp(Theta - max Theta) as B operands (hi and lo BF16 parts)
    for (int idx = tid; idx < TC_K * TC_K; idx += WS_THREADS) {
        const int y = idx / TC_K, x = idx % TC_K;
        const float psi = g.psi_shared[x * TC_K + y];
        const __nv_bfloat16 hi = __float2bfloat16_rn(psi);
        const __nv_bfloat16 lo = __float2bfloat16_rn(psi - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16 *>(sm + L::B_HI + core_offset(y, x)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(sm + L::B_LO + core_offset(y, x)) = lo;
    }
    if (tid == 0) {
        for (int s = 0; s < WS_STAGES; ++s) {
            ws_mbar_init(full0 + 8 * s, 1);   // the producer's arrival with the stage's bytes
            ws_mbar_init(empty0 + 8 * s, WS_CONS);
        }
        ws_mbar_init(mma_bar, 1);
        ws_mbar_init(old_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int n_local =
        (int)blockIdx.x < n_tiles ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;

    if (warp == 0) {
        // ---------------- producer
        constexpr int RW = (int)(sizeof(TcTileRec) / 16);   // 16-byte words of a tile record
        static_assert(RW <= 64, "a tile record is read as two words per lane");
        // the next tile's record (words lane, lane + 32) and the run state of
        // this lane's vertex, loaded one tile ahead
        uint4 ra = make_uint4(0u, 0u, 0u, 0u), rb = ra;
        int nrun = 0, ncur = 0;
        auto fetch = [&](int i) {
            const uint4 *rw = reinterpret_cast<const uint4 *>(tile_rec + ((int)blockIdx.x + i * (int)gridDim.x));
            ra = rw[lane];
            if (lane + 32 < RW)
                rb = rw[lane + 32];
            const int va = __shfl_sync(0xffffffffu, (int)ra.x, 0), nvt = __shfl_sync(0xffffffffu, (int)ra.y, 0);
            const int gg0 = __shfl_sync(0xffffffffu, (int)ra.x, 1), gg1 = __shfl_sync(0xffffffffu, (int)ra.y, 1);
            nrun = 0;
            ncur = 0;
            if (lane < nvt) {
                const int gg = gg0 == gg1 ? gg0 : g.gid[va + lane];
                const GState *gs = dr.gs + gg;
                nrun = gs->status == ST_RUNNING;
                ncur = gs->cur;
            }
        };
        if (n_local > 0)
            fetch(0);
        for (int i = 0; i < n_local; ++i) {
            const int s = i % WS_STAGES;
            if (i >= WS_STAGES && !ws_wait(empty0 + 8 * s, ((i / WS_STAGES) - 1) & 1)) {
                if (lane == 0)
                    atomicExch(err_flag, 1);
                return;
            }
            unsigned char *st = sm + s * L::STAGE;
            WsMeta &m = *reinterpret_cast<WsMeta *>(st + L::META);
            uint4 *mw = reinterpret_cast<uint4 *>(&m.rec);
            mw[lane] = ra;
            if (lane + 32 < RW)
                mw[lane + 32] = rb;
            const int va = __shfl_sync(0xffffffffu, (int)ra.x, 0), nvt = __shfl_sync(0xffffffffu, (int)ra.y, 0);
            if (lane < nvt)
                m.cur_of[lane] = nrun ? ncur : -1;
            // every running graph holds its committed messages in the same
            // buffer (LBP flips all running graphs together): read from it
            const unsigned runm = __ballot_sync(0xffffffffu, lane < nvt && nrun);
            const int buf = runm ? __shfl_sync(0xffffffffu, ncur, __ffs(runm) - 1) : 0;
            if (lane == 0)
                m.buf = buf;
            __syncwarp();
            const unsigned fb = full0 + 8 * s;
            if (lane == 0) {
                ws_expect_tx(fb, (unsigned)L::TX);   // the producer's arrival, with the bytes the copies bring
                ws_tile2d(smem_u32(st + L::UN), &maps.un, va, fb);
            }
            __syncwarp();
            // incoming rows: lane k gathers rows 4k .. 4k + 3 (rev 0 past the tile)
            {
                const int4 rv = reinterpret_cast<const int4 *>(m.rec.rev)[lane];
                ws_gather4(smem_u32(st + L::ROWS + 4 * lane * L::ROWB), &maps.in[buf], rv.x, rv.y, rv.z, rv.w, fb);
            }
            if (i + 1 < n_local)
                fetch(i + 1);   // its loads land while this warp waits for the next free stage
        }
        return;
    }

    // ---------------- consumers
    const int cw = warp - 1;                     // 0..3: vertex-field warps
    const int row = ((warp & 3) << 5) + lane;    // tensor-memory lane of this thread = its edge row
    const unsigned tmem = *tmem_slot;
    const unsigned taddr = tmem + ((unsigned)((warp & 3) * 32) << 16);
    float *SF = reinterpret_cast<float *>(sm + L::SF);
    const float floor_log = -80.0f;
    const int slot = (int)blockIdx.x & (NSUB - 1);
    unsigned phase = 0;
    bool mma_pending = false, failed = false;
    int fail_i = 0;
    int acc_g = -1;
    float acc_max = 0.0f;
    unsigned acc_cnt = 0;
    for (int i = 0; i < n_local; ++i) {
        const int s = i % WS_STAGES;
        unsigned char *st = sm + s * L::STAGE;
        const WsMeta &m = *reinterpret_cast<const WsMeta *>(st + L::META);
        const bool ok = ws_wait(full0 + 8 * s, (i / WS_STAGES) & 1);
        const int nvt = ok ? m.rec.nvt : 0;
        // 1. vertex fields S_v(x) = theta_v(x) + incoming logs, in edge order:
        //    this warp's vertices cw, cw + 4, ... summed side by side (eight
        //    independent chains instead of one vertex after another)
        {
            constexpr int VPW = TC_VMAX / WS_CONS;
            float sv[VPW];
            int rb[VPW], re[VPW];
            int maxd = 0;
#pragma unroll
            for (int j = 0; j < VPW; ++j) {
                const int vl = cw + WS_CONS * j;
                const bool in = vl < nvt;
                rb[j] = in ? (int)m.rec.rpl[vl] : 0;
                re[j] = in ? (int)m.rec.rpl[vl + 1] : 0;
                sv[j] = in ? *reinterpret_cast<const float *>(st + L::UN + swz<128>(vl, lane >> 2) + 4 * (lane & 3))
                           : 0.0f;
                maxd = max(maxd, re[j] - rb[j]);
            }
            for (int k = 0; k < maxd; ++k) {
#pragma unroll
                for (int j = 0; j < VPW; ++j)
                    if (rb[j] + k < re[j])
                        sv[j] += Store<S>::val(
                            reinterpret_cast<const S *>(st + L::ROWS + (rb[j] + k) * L::ROWB)[lane], qs);
            }
#pragma unroll
            for (int j = 0; j < VPW; ++j) {
                const int vl = cw + WS_CONS * j;
                if (vl < nvt)
                    SF[vl * TP_STRIDE + lane] = sv[j];
            }
        }
        if (ws_cons_sync_or(!ok)) {
            failed = true;
            fail_i = i;
            break;
        }
        const int ne = m.rec.ne, e0 = m.rec.e0;
        const bool has_row = row < ne;
        const int src = has_row ? m.rec.src[row] : 0;
        const int c_row = has_row ? m.cur_of[src] : -1;
        const float *svr = SF + src * TP_STRIDE;
        // 2. A operand: thread = edge row. The cavities cav(x) = S_src(x) -
        //    m_in(x) are read once into registers, group by group of 8 states
        //    in a rotated order (slot j holds group (j + row) mod 4), so the
        //    threads of a shared-memory phase mostly read different banks of
        //    the unswizzled rows; then the maximum (exact in any order) and
        //    a = exp(cav - max) per group, written as BF16 hi / lo parts at the
        //    group's columns.
        float cav[TC_K];   // cav[8 j + t]: state 8 ((j + row) mod 4) + t
#pragma unroll
        for (int j = 0; j < TC_K / 8; ++j) {
            const int q = (j + row) & 3;
            float v[8];
            if constexpr (sizeof(S) == 4) {
                ws_unpack<S>(ws_chunk<S>(st + L::ROWS, row, 2 * q), v, qs);
                ws_unpack<S>(ws_chunk<S>(st + L::ROWS, row, 2 * q + 1), v + 4, qs);
            } else {
                ws_unpack<S>(ws_chunk<S>(st + L::ROWS, row, q), v, qs);
            }
            const float4 s0 = reinterpret_cast<const float4 *>(svr)[2 * q];
            const float4 s1 = reinterpret_cast<const float4 *>(svr)[2 * q + 1];
            const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
            for (int t = 0; t < 8; ++t)
                cav[8 * j + t] = sv[t] - v[t];
        }
        float mx = -1e30f;
        if (has_row) {
            float m4[4] = {cav[0], cav[1], cav[2], cav[3]};
#pragma unroll
            for (int x = 4; x < TC_K; ++x)
                m4[x & 3] = fmaxf(m4[x & 3], cav[x]);
            mx = fmaxf(mx, fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3])));
        }
#pragma unroll
        for (int j = 0; j < TC_K / 8; ++j) {
            const int q = (j + row) & 3;
            unsigned hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                unsigned hb[2], lb[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float a = has_row ? __expf(cav[8 * j + t + u] - mx) : 0.0f;
                    const __nv_bfloat16 h = __float2bfloat16_rn(a);
                    const __nv_bfloat16 l = __float2bfloat16_rn(a - __bfloat162float(h));
                    hb[u] = __bfloat16_as_ushort(h);
                    lb[u] = __bfloat16_as_ushort(l);
                }
                hw[t / 2] = hb[0] | (hb[1] << 16);   // element x at the lower address
                lw[t / 2] = lb[0] | (lb[1] << 16);
            }
            *reinterpret_cast<uint4 *>(sm + L::A_HI + core_offset(row, 8 * q)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(sm + L::A_LO + core_offset(row, 8 * q)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        // generic-proxy reads of the rows and writes of the A operand come
        // before the async-proxy copy into the rows and the MMAs
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        ws_cons_sync();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // 3. the old rows of the tile's edges into the row region (every
        //    consumer has finished reading the incoming rows), then the MMAs
        //    from one thread: D = A_hi Psi_hi (+ A_lo Psi_hi + A_hi Psi_lo)
        if (warp == 1 && lane == 0) {
            ws_expect_tx(old_bar, (unsigned)L::TX_OLD);
            ws_tile2d(smem_u32(st + L::ROWS), &maps.old[m.buf], e0, old_bar);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                mma_bf16(tmem, make_desc(sm + L::A_HI + ks * 256, 128, 512), make_desc(sm + L::B_HI + ks * 256, 128, 512),
                         ks > 0);
            if (split) {
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    mma_bf16(tmem, make_desc(sm + L::A_LO + ks * 256, 128, 512),
                             make_desc(sm + L::B_HI + ks * 256, 128, 512), 1);
                    mma_bf16(tmem, make_desc(sm + L::A_HI + ks * 256, 128, 512),
                             make_desc(sm + L::B_LO + ks * 256, 128, 512), 1);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mma_bar));
        }
        const bool mma_ok = ws_wait(mma_bar, phase);
        const bool old_ok = ws_wait(old_bar, phase);
        if (ws_cons_sync_or(!(mma_ok && old_ok))) {
            failed = true;
            fail_i = i;
            mma_pending = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        float d[TC_K];
        {
            unsigned r[TC_K];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                         "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
                         "%28, %29, %30, %31}, [%32];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                           "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                           "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < TC_K; ++j)
                d[j] = __uint_as_float(r[j]);
        }
        // 4. epilogue: thread = row
        float r = 0.0f;
        const bool live = has_row && c_row >= 0;
        if (live) {
            const int e = e0 + row;
            float z = 0.0f;
#pragma unroll
            for (int y = 0; y < TC_K; ++y)
                z += d[y];
            S *out = (S *)msg_buf(dr, MODE == MODE_LBP ? (c_row ^ 1) : 1) + (size_t)e * TC_K;
            if constexpr (sizeof(S) == 4) {
                const float iz = __fdividef(1.0f, z);
#pragma unroll
                for (int j = 0; j < TC_K / 4; ++j) {
                    const uint4 o = *reinterpret_cast<const uint4 *>(st + L::ROWS + swz<128>(row, j));
                    const float ov[4] = {__uint_as_float(o.x), __uint_as_float(o.y), __uint_as_float(o.z),
                                         __uint_as_float(o.w)};
                    float l[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const float pn = d[4 * j + t] * iz;
                        l[t] = fmaxf(__logf(pn), floor_log);
                        r = fmaxf(r, fabsf(__expf(l[t]) - __expf(ov[t])));
                    }
                    reinterpret_cast<float4 *>(out)[j] = make_float4(l[0], l[1], l[2], l[3]);
                }
            } else {
                // BF16 words packed eight to a 16-byte store (the same words as per-state stores)
#pragma unroll
                for (int j = 0; j < TC_K / 8; ++j) {
                    const uint4 o = *reinterpret_cast<const uint4 *>(st + L::ROWS + swz<64>(row, j));
                    const unsigned ow[4] = {o.x, o.y, o.z, o.w};
                    unsigned w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        float lnew = __logf(__fdividef(d[8 * j + t], z));
                        lnew = lnew > floor_log ? lnew : floor_log;
                        const S c = Store<S>::code(lnew, qs);
                        const float pn = __expf(Store<S>::val(c, qs));
                        const unsigned short ob = (unsigned short)(ow[t >> 1] >> (16 * (t & 1)));
                        const float po = __expf(Store<S>::val(__ushort_as_bfloat16(ob), qs));
                        r = fmaxf(r, fabsf(pn - po));
                        w[t >> 1] |= (unsigned)__bfloat16_as_ushort(c) << (16 * (t & 1));
                    }
                    reinterpret_cast<uint4 *>(out)[j] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            if (MODE == MODE_CAND)
                ((float *)dr.resid)[e] = r;
            if (m.rec.gg0 != m.rec.gg1) {
                // tile spanning graphs: account the message to its own graph
                const int gg = g.gid[m.rec.va + src];
                if (r > 0.0f)
                    atomicMax(&dr.red_max[(size_t)gg * NSUB + slot], (unsigned long long)__double_as_longlong((double)r));
                if (r >= eps_in(rp, 0.0f))
                    atomicAdd(&dr.red_cnt[(size_t)gg * NSUB + slot], 1u);
            }
        }
        if (m.rec.gg0 == m.rec.gg1) {   // the same for every thread of the tile
            if (m.rec.gg0 != acc_g) {
                ws_flush(dr, acc_g, acc_max, acc_cnt, slot);
                acc_g = m.rec.gg0;
                acc_max = 0.0f;
                acc_cnt = 0;
            }
            if (live) {
                acc_max = fmaxf(acc_max, r);
                acc_cnt += (r >= eps_in(rp, 0.0f)) ? 1u : 0u;
            }
        }
        // release the stage: this warp's shared-memory reads of it (generic
        // proxy) come before the copies that will refill it (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0)
            ws_arrive(empty0 + 8 * s);
        // the next tile's MMAs overwrite tensor memory only after the consumer
        // barrier of its A operand, which every thread reaches after this read
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    ws_flush(dr, acc_g, acc_max, acc_cnt, slot);
    if (failed) {
        if (warp == 1 && lane == 0)
            atomicExch(err_flag, 1);
        // the MMAs and copies of the failed tile and the copies of staged tiles
        // may still be in flight: wait for them (bounded) before the CTA leaves
        if (mma_pending) {
            ws_wait(mma_bar, phase);
            ws_wait(old_bar, phase);
        }
        for (int q = fail_i; q < n_local && q < fail_i + WS_STAGES; ++q)
            ws_wait(full0 + 8 * (q % WS_STAGES), (q / WS_STAGES) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    ws_cons_sync();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

template <typename S> constexpr size_t ws_smem_bytes() { return (size_t)WsLayout<S>::TOTAL + 1024; }

// CTAs of the warp-specialised kernel per SM x SMs, once per device. Shared
// memory is the limit (registers allow more): the SM's shared memory over the
// CTA's dynamic bytes plus the per-block reservation.
template <typename S, int MODE> int ws_grid_cap()
{
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    std::call_once(once[dev], [&] {
        cudaFuncSetAttribute(k_potts_ws<S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem_bytes<S>());
        int sms = 0, per_sm = 0, reserved = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        const int nb = per_sm / ((int)ws_smem_bytes<S>() + reserved);
        cached[dev] = std::min(std::max(nb, 1), 4) * std::max(sms, 1);
    });
    return cached[dev];
}

// cuTensorMapEncodeTiled from the driver (looked up once).
using WsEncodeFn = PFN_cuTensorMapEncodeTiled_v12000;
static WsEncodeFn ws_encode_fn()
{
    static WsEncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<WsEncodeFn>(p);
    });
    return fn;
}

// A [rows x row_bytes] row-major tensor at base with a box of box_rows whole rows.
static bool ws_map2d(CUtensorMap *map, CUtensorMapDataType dt, const void *base, unsigned long long rows,
                     int row_bytes, unsigned box_rows, CUtensorMapSwizzle swizzle)
{
    const WsEncodeFn fn = ws_encode_fn();
    if (!fn || !base)
        return false;
    const int esz = dt == CU_TENSOR_MAP_DATA_TYPE_FLOAT32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)(row_bytes / esz), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {(cuuint32_t)(row_bytes / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename S> static bool ws_make_maps(const DevGraph &g, const DevRun &dr, WsMaps &mp)
{
    const CUtensorMapDataType dt = sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUtensorMapSwizzle sw = sizeof(S) == 4 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const int rb = TC_K * (int)sizeof(S);
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
        ok = ok && ws_map2d(&mp.in[b], dt, dr.msg[b], (unsigned long long)g.M, rb, 1, CU_TENSOR_MAP_SWIZZLE_NONE);
        ok = ok && ws_map2d(&mp.old[b], dt, dr.msg[b], (unsigned long long)g.M, rb, TC_ROWS, sw);
    }
    ok = ok && ws_map2d(&mp.un, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g.unary, (unsigned long long)g.n, TC_K * 4, TC_VMAX,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    return ok;
}

// false when the tensor maps cannot be made (the caller runs the single-stage kernel)
template <typename S, int MODE>
static bool launch_ws_t(const DevGraph &g, const DevRun &dr, const RunParams &rp, const TcTileRec *tile_rec,
                        int n_tiles, int split, int *err_flag, cudaStream_t s)
{
    WsMaps maps;
    if (!ws_make_maps<S>(g, dr, maps))
        return false;
    const int grid = std::min(n_tiles, ws_grid_cap<S, MODE>());
    k_potts_ws<S, MODE><<<grid, WS_THREADS, ws_smem_bytes<S>(), s>>>(g, dr, rp, tile_rec, n_tiles, split, err_flag,
                                                                     maps);
    return true;
}

static void prepare_ws()
{
    ws_grid_cap<float, MODE_LBP>();
    ws_grid_cap<float, MODE_CAND>();
    ws_grid_cap<__nv_bfloat16, MODE_LBP>();
    ws_grid_cap<__nv_bfloat16, MODE_CAND>();
}

size_t potts_tc_pipe_smem_bytes() { return sizeof(TcPipeShared) + 1024; }

size_t potts_tc_smem_bytes() { return sizeof(TcShared) + 1024; }

template <bool TC> static void set_tc_attr()
{
    const int sm = (int)potts_tc_smem_bytes();
    cudaFuncSetAttribute(k_potts_tc<float, MODE_LBP, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_potts_tc<float, MODE_CAND, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_potts_tc<__nv_bfloat16, MODE_LBP, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_potts_tc<__nv_bfloat16, MODE_CAND, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

void prepare_potts_tc()
{
    prepare_ws();
    set_tc_attr<true>();
    set_tc_attr<false>();
    const int sm = (int)potts_tc_pipe_smem_bytes();
    cudaFuncSetAttribute(k_potts_tc_pipe<MODE_LBP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_potts_tc_pipe<MODE_CAND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <bool TC>
static void launch_tc_t(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode,
                        const int *tile_v, int n_tiles, int split, int *err_flag, cudaStream_t s)
{
    if constexpr (!TC) {
        if (dtype == DT_F32 && g.k == TC_K) {
            // CUDA-core path: pipelined form, 3 CTAs per SM (two staging buffers
            // per CTA; 80 us against 98 us per 261,120-message launch). The
            // tensor-core path keeps 4 CTAs per SM without the second stage
            // (57 us against 66 us).
            const int grid = n_tiles < 152 * 3 ? n_tiles : 152 * 3;
            const size_t sm = potts_tc_pipe_smem_bytes();
            if (mode == MODE_LBP)
                k_potts_tc_pipe<MODE_LBP, TC><<<grid, TC_THREADS, sm, s>>>(g, dr, rp, tile_v, n_tiles, split,
                                                                          err_flag);
            else
                k_potts_tc_pipe<MODE_CAND, TC><<<grid, TC_THREADS, sm, s>>>(g, dr, rp, tile_v, n_tiles, split,
                                                                           err_flag);
            return;
        }
    }
    const int grid = n_tiles < 152 * 4 ? n_tiles : 152 * 4;
    const size_t sm = potts_tc_smem_bytes();
    if (dtype == DT_BF16) {
        if (mode == MODE_LBP)
            k_potts_tc<__nv_bfloat16, MODE_LBP, TC><<<grid, TC_THREADS, sm, s>>>(g, dr, rp, tile_v, n_tiles, split,
                                                                               err_flag);
        else
            k_potts_tc<__nv_bfloat16, MODE_CAND, TC><<<grid, TC_THREADS, sm, s>>>(g, dr, rp, tile_v, n_tiles, split,
                                                                                err_flag);
    } else {
        if (mode == MODE_LBP)
            k_potts_tc<float, MODE_LBP, TC><<<grid, TC_THREADS, sm, s>>>(g, dr, rp, tile_v, n_tiles, split, err_flag);
        else
            k_potts_tc<float, MODE_CAND, TC><<<grid, TC_THREADS, sm, s>>>(g, dr, rp, tile_v, n_tiles, split, err_flag);
    }
}

void launch_potts_tc(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode,
                     const int *tile_v, const TcTileRec *tile_rec, int n_tiles, int path, int *err_flag,
                     cudaStream_t s)
{
    if (n_tiles == 0)
        return;
    if (path == 1) {
        launch_tc_t<false>(dtype, g, dr, rp, mode, tile_v, n_tiles, 0, err_flag, s);
        return;
    }
    // k = 32 (every state present in each row) and boxes within the tensors:
    // the warp-specialised form; otherwise, or when the driver cannot encode
    // its tensor maps, the single-stage kernel
    const int split = path == 3;
    bool done = false;
    if (g.k == TC_K && tile_rec && g.M >= TC_ROWS && g.n >= TC_VMAX) {
        if (dtype == DT_F32)
            done = mode == MODE_LBP ? launch_ws_t<float, MODE_LBP>(g, dr, rp, tile_rec, n_tiles, split, err_flag, s)
                                    : launch_ws_t<float, MODE_CAND>(g, dr, rp, tile_rec, n_tiles, split, err_flag, s);
        else if (dtype == DT_BF16)
            done = mode == MODE_LBP
                       ? launch_ws_t<__nv_bfloat16, MODE_LBP>(g, dr, rp, tile_rec, n_tiles, split, err_flag, s)
                       : launch_ws_t<__nv_bfloat16, MODE_CAND>(g, dr, rp, tile_rec, n_tiles, split, err_flag, s);
    }
    if (!done)
        launch_tc_t<true>(dtype, g, dr, rp, mode, tile_v, n_tiles, split, err_flag, s);
}

}  // namespace bpg
