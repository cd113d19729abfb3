// bp_lbp_run_noalloc: synchronous loopy BP on one binary Ising graph that
// allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// framework whose caching allocator has already reserved the device memory,
// code on a latency-critical path where cudaMalloc/cudaFree would synchronise
// the device, or plug-ins that must not change the process's allocation state.
// They pass their inputs and outputs in device memory they own; the scratch
// this run needs (two message buffers, exp(-2 beta), unary log-odds, the
// per-run state and the convergence reductions) lives in one file-scope
// static device array below. The CUDA runtime loads device code lazily, so
// the first call made on a device loads it (scratch_for_current_device loads
// every kernel the call launches and looks up the array); from then on the
// device holds the array until the process exits, and no call allocates
// anything.
#include "bp_gb300.h"
#include "bp_internal.cuh"
#include "bp_launch.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

using namespace bpg;

namespace {

// Capacity of the static scratch.
constexpr int64_t NA_MAX_EDGES = 1 << 18;   // directed messages (a 256x256 grid has 261,120)
constexpr int32_t NA_MAX_VARS = 1 << 17;    // vertices

// Byte offsets of the scratch regions (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_MSG0 = 0;
constexpr size_t OFF_MSG1 = align256(OFF_MSG0 + sizeof(float) * NA_MAX_EDGES);
constexpr size_t OFF_Q32 = align256(OFF_MSG1 + sizeof(float) * NA_MAX_EDGES);
constexpr size_t OFF_UD32 = align256(OFF_Q32 + sizeof(float) * NA_MAX_EDGES);
constexpr size_t OFF_UD64 = align256(OFF_UD32 + sizeof(float) * NA_MAX_VARS);
constexpr size_t OFF_GID = align256(OFF_UD64 + sizeof(double) * NA_MAX_VARS);
constexpr size_t OFF_GOFF = align256(OFF_GID + sizeof(int32_t) * NA_MAX_VARS);   // gv_off[2], ge_off[2]
constexpr size_t OFF_GS = align256(OFF_GOFF + sizeof(int32_t) * 4);
constexpr size_t OFF_REDMAX = align256(OFF_GS + sizeof(GState));
constexpr size_t OFF_REDCNT = align256(OFF_REDMAX + sizeof(unsigned long long) * NSUB);
constexpr size_t OFF_RUNNING = align256(OFF_REDCNT + sizeof(unsigned int) * NSUB);
constexpr size_t OFF_ERR = OFF_RUNNING + 16;
constexpr size_t NA_SCRATCH_BYTES = align256(OFF_ERR + 16);

// The scratch itself: about 5.0 MiB, shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, filled on the first call
// made with that device current.
constexpr int NA_MAX_DEVICES = 64;
unsigned char *g_scratch_addr[NA_MAX_DEVICES];
std::mutex g_scratch_mu;

enum : unsigned { NA_BAD_GRAPH = 1u, NA_NONFINITE = 2u };

// Checks the CSR and the potentials; every index is range-checked before it
// is used, and a violation sets a bit in *err instead of touching memory.
// Thread 0 also checks row_ptr[0] == 0 and row_ptr[n] == M; the other threads
// do not wait for that check, which is safe because each thread checks its
// own row range against [0, M] before reading col or rev, so a wrong first or
// last entry is reported without any read outside the arrays.
__global__ void k_na_validate(int32_t n, int32_t M, const int32_t *row_ptr, const int32_t *col,
                              const int32_t *rev, const float *unary, const float *beta, unsigned *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (row_ptr[0] != 0 || row_ptr[n] != M))
        atomicOr(err, NA_BAD_GRAPH);
    if (i >= n)
        return;
    if (!isfinite(unary[2 * i]) || !isfinite(unary[2 * i + 1]))
        atomicOr(err, NA_NONFINITE);
    const int beg = row_ptr[i], end = row_ptr[i + 1];
    if (beg < 0 || end > M || beg > end) {
        atomicOr(err, NA_BAD_GRAPH);
        return;
    }
    for (int e = beg; e < end; ++e) {
        const int j = col[e], r = rev[e];
        if (j < 0 || j >= n || j == i || r < 0 || r >= M || r == e) {
            atomicOr(err, NA_BAD_GRAPH);
            continue;
        }
        const int jb = row_ptr[j], je = row_ptr[j + 1];
        if (r < jb || r >= je || col[r] != i || rev[r] != e)
            atomicOr(err, NA_BAD_GRAPH);
        if (!isfinite(beta[e]) || beta[r] != beta[e])
            atomicOr(err, NA_NONFINITE);
    }
}

// Derived potentials and the starting state (uniform messages: log-odds 0).
__global__ void k_na_prepare(int32_t n, int32_t M, const float *unary, const float *beta, unsigned char *sc)
{
    float *msg0 = (float *)(sc + OFF_MSG0);
    float *msg1 = (float *)(sc + OFF_MSG1);
    float *q32 = (float *)(sc + OFF_Q32);
    float *ud32 = (float *)(sc + OFF_UD32);
    double *ud64 = (double *)(sc + OFF_UD64);
    int32_t *gid = (int32_t *)(sc + OFF_GID);
    const int stride = gridDim.x * blockDim.x;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M; e += stride) {
        const double q = exp(-2.0 * (double)beta[e]);
        q32[e] = (float)fmin(fmax(q, 1e-30), 1e30);
        msg0[e] = 0.0f;
        msg1[e] = 0.0f;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double d = (double)unary[2 * i + 1] - (double)unary[2 * i];
        ud64[i] = d;
        ud32[i] = (float)d;
        gid[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int32_t *goff = (int32_t *)(sc + OFF_GOFF);
        goff[0] = 0;
        goff[1] = n;
        goff[2] = 0;
        goff[3] = M;
        GState *gs = (GState *)(sc + OFF_GS);
        gs->status = ST_RUNNING;
        gs->rounds = 0;
        gs->cur = 0;
        gs->k_sel = 0;
        gs->thr = 0;
        gs->always = 0;
        gs->n_prev = 0;
        gs->committed = 0;
        gs->evals = 0;
        gs->full_evals = 0;
        gs->full_nodes = 0;
        gs->final_maxr = 0.0;
        gs->final_cnt = 0;
        *(int32_t *)(sc + OFF_RUNNING) = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x < NSUB) {
        ((unsigned long long *)(sc + OFF_REDMAX))[threadIdx.x] = 0ull;
        ((unsigned int *)(sc + OFF_REDCNT))[threadIdx.x] = 0u;
    }
}

int na_fail(int code, const std::string &msg)
{
    set_last_error(msg);
    return code;
}

// Device address of the scratch for the current device (set up once per device).
int scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return na_fail(BP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES)
        return na_fail(BP_ERR_UNSUPPORTED, "device ordinal beyond the scratch table");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        // set-up: load the kernels this entry point launches (so that later
        // calls load nothing) and look up the array, which loads its module
        e = preload_lbp_f32_kernels();
        if (e != cudaSuccess)
            return na_fail(BP_ERR_CUDA, std::string("kernel load: ") + cudaGetErrorString(e));
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k_na_validate);
        if (e == cudaSuccess)
            e = cudaFuncGetAttributes(&fa, k_na_prepare);
        if (e != cudaSuccess)
            return na_fail(BP_ERR_CUDA, std::string("kernel load: ") + cudaGetErrorString(e));
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(BP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return BP_OK;
}

}  // namespace

extern "C" {

int bp_lbp_run_noalloc(int32_t n_vars, int64_t n_dir_edges, const int32_t *row_ptr, const int32_t *col,
                       const int32_t *rev, const float *unary_log, const float *beta, double eps,
                       int32_t max_rounds, double *beliefs, int32_t *rounds_out, int32_t *converged_out,
                       void *cuda_stream)
{
    if (n_vars < 1 || n_dir_edges < 0 || !row_ptr || !unary_log || !beliefs ||
        (n_dir_edges > 0 && (!col || !rev || !beta)))
        return na_fail(BP_ERR_INVALID_ARG, "bp_lbp_run_noalloc: NULL pointer or negative size");
    if (n_vars > NA_MAX_VARS || n_dir_edges > NA_MAX_EDGES)
        return na_fail(BP_ERR_UNSUPPORTED,
                       "bp_lbp_run_noalloc: graph exceeds the static scratch (at most " +
                           std::to_string(NA_MAX_VARS) + " vertices and " + std::to_string(NA_MAX_EDGES) +
                           " directed edges)");
    if (!(eps > 0.0) || !std::isfinite(eps) || max_rounds < 0)
        return na_fail(BP_ERR_INVALID_ARG, "bp_lbp_run_noalloc: eps must be positive, max_rounds >= 0");
    // An error that earlier CUDA work of this thread left pending belongs to
    // that work: consume it so that the launch checks below see only ours.
    (void)cudaGetLastError();
    unsigned char *sc = nullptr;
    int rc = scratch_for_current_device(&sc);
    if (rc != BP_OK)
        return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int32_t n = n_vars, M = (int32_t)n_dir_edges;
    unsigned *d_err = (unsigned *)(sc + OFF_ERR);
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), s);
    if (e != cudaSuccess)
        return na_fail(BP_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_na_validate<<<(n + 255) / 256, 256, 0, s>>>(n, M, row_ptr, col, rev, unary_log, beta, d_err);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return na_fail(BP_ERR_CUDA, std::string("validation launch: ") + cudaGetErrorString(e));
    unsigned h_err = 0;
    e = cudaMemcpyAsync(&h_err, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return na_fail(BP_ERR_CUDA, std::string("validation: ") + cudaGetErrorString(e));
    if (h_err & NA_BAD_GRAPH)
        return na_fail(BP_ERR_BAD_GRAPH, "bp_lbp_run_noalloc: invalid CSR or reverse-edge index");
    if (h_err & NA_NONFINITE)
        return na_fail(BP_ERR_NONFINITE, "bp_lbp_run_noalloc: non-finite or asymmetric potentials");

    const int pb = std::min((std::max(n, M) + 255) / 256, 152 * 8);
    k_na_prepare<<<pb, 256, 0, s>>>(n, M, unary_log, beta, sc);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return na_fail(BP_ERR_CUDA, std::string("set-up launch: ") + cudaGetErrorString(e));

    DevGraph g;
    memset(&g, 0, sizeof(g));
    g.n = n;
    g.k = 2;
    g.G = 1;
    g.M = M;
    g.epm = 1;
    g.qscale = 1.0f;
    // the caller's rev may sit at any address; the scratch arrays are aligned
    g.vec_ok = ((reinterpret_cast<uintptr_t>(rev) & 15u) == 0) ? 1 : 0;
    g.row_ptr = row_ptr;
    g.col = col;
    g.rev = rev;
    g.gid = (const int32_t *)(sc + OFF_GID);
    g.gv_off = (const int32_t *)(sc + OFF_GOFF);
    g.ge_off = (const int32_t *)(sc + OFF_GOFF) + 2;
    g.pair_kind = BP_PAIR_ISING_BETA;
    g.unary = unary_log;
    g.udiff32 = (const float *)(sc + OFF_UD32);
    g.udiff64 = (const double *)(sc + OFF_UD64);
    g.q32 = (const float *)(sc + OFF_Q32);
    DevRun dr;
    memset(&dr, 0, sizeof(dr));
    dr.msg[0] = sc + OFF_MSG0;
    dr.msg[1] = sc + OFF_MSG1;
    dr.gs = (GState *)(sc + OFF_GS);
    dr.red_max = (unsigned long long *)(sc + OFF_REDMAX);
    dr.red_cnt = (unsigned int *)(sc + OFF_REDCNT);
    dr.n_running = (int32_t *)(sc + OFF_RUNNING);
    dr.beliefs = beliefs;
    RunParams rp;
    memset(&rp, 0, sizeof(rp));
    rp.schedule = SCHED_LBP;
    rp.max_rounds = max_rounds;
    rp.eps = eps;
    rp.low_p = 1.0;
    rp.high_p = 1.0;
    rp.variant = 1;
    {
        float f = (float)eps;   // smallest float >= eps
        if ((double)f < eps)
            f = std::nextafter(f, 3.0e38f);
        rp.eps_f = f;
    }

    // Rounds are launched directly; the host reads the running flag every
    // `chunk` rounds (rounds after convergence are no-ops on the device).
    int32_t running = 1;
    int64_t launched = 0;
    int chunk = 2;
    while (running > 0) {
        for (int r = 0; r < chunk; ++r) {
            launch_eval(DT_F32, g, dr, rp, MODE_LBP, 0, 4, s);
            launch_decide(g, dr, rp, s);
        }
        launched += chunk;
        // a failed launch stops here, before its zeroed reductions could be
        // read as convergence by the next poll
        if ((e = cudaGetLastError()) != cudaSuccess)
            return na_fail(BP_ERR_CUDA, std::string("round launch: ") + cudaGetErrorString(e));
        e = cudaMemcpyAsync(&running, dr.n_running, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return na_fail(BP_ERR_CUDA, std::string("round loop: ") + cudaGetErrorString(e));
        // every graph stops after at most max_rounds + 1 evaluations, so a
        // running graph past that point is a broken invariant, not a CUDA error
        if (running > 0 && launched > (int64_t)max_rounds + 1)
            return na_fail(BP_ERR_INTERNAL, "bp_lbp_run_noalloc: round loop did not terminate");
        chunk = std::min(chunk * 2, 64);
    }
    launch_beliefs(DT_F32, g, dr, 4, s);
    GState st;
    if ((e = cudaGetLastError()) != cudaSuccess)
        return na_fail(BP_ERR_CUDA, std::string("beliefs launch: ") + cudaGetErrorString(e));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&st, dr.gs, sizeof(GState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return na_fail(BP_ERR_CUDA, std::string("beliefs: ") + cudaGetErrorString(e));
    if (rounds_out)
        *rounds_out = st.rounds;
    if (converged_out)
        *converged_out = st.status == ST_CONVERGED;
    return BP_OK;
}

}  // extern "C"
