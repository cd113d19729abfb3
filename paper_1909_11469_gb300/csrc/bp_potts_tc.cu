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

#include <cuda_bf16.h>

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
                     const int *tile_v, int n_tiles, int path, int *err_flag, cudaStream_t s)
{
    if (n_tiles == 0)
        return;
    if (path == 1)
        launch_tc_t<false>(dtype, g, dr, rp, mode, tile_v, n_tiles, 0, err_flag, s);
    else
        launch_tc_t<true>(dtype, g, dr, rp, mode, tile_v, n_tiles, path == 3, err_flag, s);
}

}  // namespace bpg
