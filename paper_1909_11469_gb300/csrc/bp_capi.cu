// Runtime and C ABI of libbp_gb300: graph validation and upload, potentials,
// the CUDA-graph-captured round loop of Algorithm 1, beliefs and statistics.
#include "bp_gb300.h"
#include "bp_internal.cuh"
#include "bp_launch.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace bpg;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();   // clear a sticky-free error so the next call starts clean
    if (e == cudaErrorMemoryAllocation)
        return fail(BP_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    return fail(BP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BP_CK(call)                                 \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess)                      \
            return cuda_fail(_e, #call);            \
    } while (0)

template <typename T> int dalloc(T **p, size_t count)
{
    *p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    return BP_OK;
}

template <typename T> void dfree(T *&p)
{
    if (p)
        cudaFree((void *)p);
    p = nullptr;
}

struct CachedGraph {
    RunParams rp;
    int dtype, rounds, kp, epm;
    int64_t kernels;                    // kernel nodes in the graph
    cudaGraphExec_t exec;
};

void destroy_cached(CachedGraph &c) { cudaGraphExecDestroy(c.exec); }

// Process-wide table of tuned binary-update mappings (bp_autotune), keyed by
// size class.
std::mutex g_tune_mu;
std::map<uint32_t, int32_t> g_tune_table;

int log2_floor(int64_t v)
{
    int b = 0;
    while (v > 1) {
        v >>= 1;
        ++b;
    }
    return b;
}

}  // namespace

void bpg::set_last_error(const std::string &msg) { g_last_error = msg; }

struct bp_graph {
    int32_t n = 0, k = 0, G = 0;
    int64_t M = 0;
    int dev = 0;
    int kp = 32;
    std::vector<int32_t> h_rev, h_gv_off, h_ge_off;
    std::vector<int32_t> h_col, h_src;   // destination and source vertex of every directed edge
    // structure
    int32_t *d_row_ptr = nullptr, *d_col = nullptr, *d_rev = nullptr, *d_gid = nullptr;
    int32_t *d_gv_off = nullptr, *d_ge_off = nullptr;
    // potentials
    int pair_kind = -1;
    bool has_pot = false;
    float qscale = 1.0f;   // Q16 log-odds step: 2 max|beta| / 32767
    float bscale = 1.0f;   // BF16 (binary Ising) log-odds per unit of log2 of the word: 2 max|beta| / 250
    int32_t sel_smem_bytes = 0;   // staged keys of the largest graph, capped
    float *d_unary = nullptr, *d_udiff32 = nullptr, *d_q32 = nullptr, *d_pair = nullptr,
          *d_psi_shared = nullptr;
    int32_t *d_kpresent = nullptr;   // present states per vertex, when some state is absent
    double *d_udiff64 = nullptr, *d_q64 = nullptr;
    // run buffers
    int buf_dtype = -1;
    int buf_epm = 0;
    void *d_msg[3] = {nullptr, nullptr, nullptr};   // the third: fused RnBP rounds (lazy)
    void *d_resid = nullptr, *d_vres = nullptr;
    int8_t *d_level = nullptr;
    int2 *d_lvl_list = nullptr;                 // Residual Splash level lists (lazy)
    int32_t *d_lvl_cnt = nullptr;
    double *d_graph_p = nullptr;   // per-graph parallelism (bp_set_graph_parallelism)
    bool graph_p_set = false;
    int32_t max_deg = 0;           // largest vertex degree (size class, mapping heuristic)
    GState *d_gs = nullptr;
    unsigned long long *d_red_max = nullptr;
    unsigned int *d_red_cnt = nullptr;
    unsigned int *d_red_commit = nullptr;
    unsigned int *d_red_commit_lo = nullptr;
    int32_t *d_running = nullptr;
    int32_t *d_queue = nullptr;
    int32_t max_graph_vertices = 0;
    int32_t max_graph_edges = 0;
    int32_t sel_plan[4][6];          // per message dtype: RBP CTAs, bytes, grid flag; RS the same
    bool sel_planned[4] = {false, false, false, false};
    // grid-wide selection buffers (allocated when a plan picks the grid kernels)
    GSelState *d_gsel = nullptr;
    unsigned int *d_gsel_hist = nullptr;
    int32_t *d_gsel_tie = nullptr, *d_chunk_off = nullptr;
    int32_t n_chunks_rbp = 0, n_chunks_rs = 0;
    // tensor-core tiles of consecutive vertices (<= 128 out-edges, <= 32 vertices)
    int32_t *d_tc_tiles = nullptr;
    TcTileRec *d_tc_rec = nullptr;   // one static record per tile
    int32_t n_tc_tiles = 0;
    bool tc_tiles_ok = false;
    int32_t *d_err = nullptr;
    PotCheck *d_potcheck = nullptr;   // checks of the device-side Ising potentials
    int32_t pot_bufs_kind = -1;       // pair kind whose potential buffers are allocated
    // warp tiles of the streamed update (mapping 6), n_wtiles + 1 records; 0
    // tiles when a vertex has more than STREAM_WT out-edges
    int4 *d_wtiles = nullptr;
    int4 *d_ctiles = nullptr;  // commit records of the warp tiles {e0, e1, graph, graph's e0}
    uint32_t *d_eps_words = nullptr;   // RnBP eps flag words, 4 per warp tile (lazy)
    int32_t n_wtiles = 0;
    bool wtiles_ok = false;
    uint32_t *d_trace = nullptr;
    size_t trace_alloc_words = 0;
    double *d_beliefs = nullptr;
    int32_t *h_running = nullptr;   // pinned
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_pt0 = nullptr, ev_pt1 = nullptr;
    std::vector<cudaEvent_t> prof_events;   // profile mode: 4 per round of a chunk
    std::vector<CachedGraph> cache;
    // last result
    bool has_result = false;
    int res_dtype = 0;
    int res_schedule = 0;
    int32_t trace_rounds = 0;
    int32_t trace_words = 0;
    std::vector<bp_run_stats> last_stats;
    bp_profile last_profile;
};

namespace {

void clear_cache(bp_graph *g)
{
    for (auto &c : g->cache)
        destroy_cached(c);
    g->cache.clear();
}

void free_run_buffers(bp_graph *g)
{
    clear_cache(g);
    dfree(g->d_msg[0]);
    dfree(g->d_msg[1]);
    dfree(g->d_msg[2]);
    dfree(g->d_resid);
    dfree(g->d_vres);
    g->buf_dtype = -1;
}

// Binary Ising messages are stored as one log-odds value, others as k logs.
int epm_of(const bp_graph *g) { return (g->k == 2 && g->pair_kind == BP_PAIR_ISING_BETA) ? 1 : g->k; }

// Size class of a handle for a schedule and storage format: mean vertices
// per graph and graph count (log2 buckets), largest degree (<= 4, <= 8, more).
uint32_t size_class(const bp_graph *g, int schedule, int dtype)
{
    const int64_t per = std::max<int64_t>(1, (int64_t)g->n / std::max(g->G, 1));
    const uint32_t nb = (uint32_t)log2_floor(per), gb = (uint32_t)log2_floor(g->G);
    const uint32_t db = g->max_deg <= 4 ? 0u : (g->max_deg <= 8 ? 1u : 2u);
    return (uint32_t)schedule | ((uint32_t)dtype << 2) | (nb << 4) | (gb << 9) | (db << 14);
}

// Binary update mapping of a run: the requested one, else the tuned one of the
// handle's size class, else thread per vertex with prefetched gathers for
// graphs of degree <= 4 (every vertex's edges held in registers) and the plain
// thread-per-vertex form otherwise. Table values: mapping in bits 0-7, tuned
// selection path in bits 8-15.
int32_t resolve_variant(const bp_graph *g, int schedule, int dtype, int32_t requested)
{
    if (requested != 0)
        return requested;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_table.find(size_class(g, schedule, dtype));
        if (it != g_tune_table.end())
            return it->second & 0xff;
    }
    if (dtype == DT_F64)
        return 1;
    // RnBP rounds commit inside the streamed update (no commit kernel), which
    // wins on low-degree grids too: 1000x1000 grid batch run 55.3 against
    // 84.6 ms with the prefetching mapping and its commit kernel
    if (schedule == BP_RNBP && g->wtiles_ok)
        return 6;
    if (g->max_deg <= 4)
        return 4;
    return g->wtiles_ok ? 6 : 1;
}

// Selection path of a run: the requested one, else the tuned one of the
// handle's size class (0 when none: the planner's estimate decides).
int32_t resolve_select_path(const bp_graph *g, int schedule, int dtype, int32_t requested)
{
    if (requested != 0)
        return requested;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_table.find(size_class(g, schedule, dtype));
    return it != g_tune_table.end() ? (it->second >> 8) & 0xff : 0;
}

// BF16 code scale of Ising potentials with max |beta| = bmax: the smallest
// power of two >= 2 bmax / 250, so every |u| <= 2 bmax has |u| / b <= 250 and
// the scaling by b and 1/b is exact.
float bf16_scale(double bmax)
{
    int ex = 0;
    const double m = std::frexp(2.0 * bmax / 250.0, &ex);   // 2 bmax / 250 = m 2^ex, m in [0.5, 1)
    return (float)std::ldexp(1.0, m == 0.5 ? ex - 1 : ex);
}

// Scale of the run's 16-bit storage (DevGraph::qscale).
float storage_scale(const bp_graph *g, int dtype)
{
    if (dtype == DT_Q16)
        return g->qscale;
    if (dtype == DT_BF16 && epm_of(g) == 1)
        return g->bscale;
    return 0.0f;
}

DevGraph dev_graph(const bp_graph *g, int dtype)
{
    DevGraph d;
    d.n = g->n;
    d.k = g->k;
    d.G = g->G;
    d.M = (int32_t)g->M;
    d.epm = epm_of(g);
    d.qscale = storage_scale(g, dtype);
    d.vec_ok = 1;   // every device array of a handle comes from cudaMalloc (256-byte aligned)
    d.sel_smem_bytes = g->sel_smem_bytes;
    d.max_ge = g->max_graph_edges;
    d.max_gv = g->max_graph_vertices;
    d.sel_c[0] = d.sel_c[1] = 1;
    d.sel_dyn[0] = d.sel_dyn[1] = 0;
    d.sel_grid[0] = d.sel_grid[1] = 0;
    d.row_ptr = g->d_row_ptr;
    d.col = g->d_col;
    d.rev = g->d_rev;
    d.gid = g->d_gid;
    d.gv_off = g->d_gv_off;
    d.ge_off = g->d_ge_off;
    d.pair_kind = g->pair_kind;
    d.unary = g->d_unary;
    d.udiff32 = g->d_udiff32;
    d.udiff64 = g->d_udiff64;
    d.q32 = g->d_q32;
    d.q64 = g->d_q64;
    d.pair = g->d_pair;
    d.psi_shared = g->d_psi_shared;
    d.kpresent = g->d_kpresent;
    d.wtiles = g->d_wtiles;
    d.ctiles = g->d_ctiles;
    d.n_wtiles = g->n_wtiles;
    return d;
}

DevRun dev_run(const bp_graph *g)
{
    DevRun r;
    r.msg[0] = g->d_msg[0];
    r.msg[1] = g->d_msg[1];
    r.msg[2] = g->d_msg[2];
    r.resid = g->d_resid;
    r.vres = g->d_vres;
    r.level = g->d_level;
    r.gs = g->d_gs;
    r.red_max = g->d_red_max;
    r.red_cnt = g->d_red_cnt;
    r.red_commit = g->d_red_commit;
    r.red_commit_lo = g->d_red_commit_lo;
    r.n_running = g->d_running;
    r.trace = g->d_trace;
    r.beliefs = g->d_beliefs;
    r.queue = g->d_queue;
    r.lvl_list = g->d_lvl_list;
    r.lvl_cnt = g->d_lvl_cnt;
    r.graph_p = g->graph_p_set ? g->d_graph_p : nullptr;
    r.err = g->d_err;
    r.eps_words = g->d_eps_words;
    r.gsel = g->d_gsel;
    r.gsel_hist = g->d_gsel_hist;
    r.gsel_tie = g->d_gsel_tie;
    r.chunk_off = g->d_chunk_off;
    r.n_chunks_rbp = g->n_chunks_rbp;
    r.n_chunks_rs = g->n_chunks_rs;
    return r;
}

// Selection shape of a run: the cluster plan of the handle for this storage
// format and the grid-wide flags the run chose (bit 0 RBP, bit 1 RS), and the
// cluster size of the splash sweep.
void apply_select_plan(const bp_graph *g, int dtype, int sel_grid_bits, DevGraph &dg)
{
    if (g->sel_planned[dtype]) {
        dg.sel_c[0] = g->sel_plan[dtype][0];
        dg.sel_dyn[0] = g->sel_plan[dtype][1];
        dg.sel_c[1] = g->sel_plan[dtype][3];
        dg.sel_dyn[1] = g->sel_plan[dtype][4];
    }
    dg.sel_grid[0] = sel_grid_bits & 1;
    dg.sel_grid[1] = (sel_grid_bits >> 1) & 1;
}

size_t dtype_size(int dt) { return dt == DT_F64 ? 8 : (dt == DT_F32 ? 4 : 2); }   // BF16, Q16: 2

// Elements appended to the arrays the streamed update reads with bulk copies
// (rev, row_ptr, exp(-2 beta), unary log-odds, messages): a copy starts at the
// 16-byte block of a tile's first element and ends at the block of its last,
// so it may read up to 15 bytes past an array's last element.
constexpr size_t PAD = 16;

int ensure_msg_buffers(bp_graph *g, int dtype)
{
    if (g->buf_dtype == dtype && g->buf_epm == epm_of(g))
        return BP_OK;
    free_run_buffers(g);
    g->buf_epm = epm_of(g);
    size_t elems = (size_t)g->M * (size_t)g->buf_epm;
    size_t es = dtype_size(dtype);
    size_t rs = dtype == DT_F64 ? 8 : 4;
    int rc;
    for (int b = 0; b < 2; ++b) {
        // (+ PAD elements: the streamed update copies whole 16-byte blocks)
        if ((rc = dalloc((char **)&g->d_msg[b], (elems + PAD) * es)) != BP_OK)
            return rc;
    }
    if ((rc = dalloc((char **)&g->d_resid, (size_t)g->M * rs)) != BP_OK)
        return rc;
    if ((rc = dalloc((char **)&g->d_vres, (size_t)g->n * rs)) != BP_OK)
        return rc;
    g->buf_dtype = dtype;
    return BP_OK;
}

int validate_and_upload(bp_graph *g, int32_t n_graphs, const int64_t *gvo, int32_t n, int32_t k, int64_t M,
                        const int64_t *row_ptr, const int32_t *col, const int32_t *rev)
{
    if (n < 0 || M < 0 || n_graphs < 1)
        return fail(BP_ERR_INVALID_ARG, "negative size or no graph");
    if (k < 2 || k > 128)
        return fail(BP_ERR_UNSUPPORTED, "n_states must be in [2, 128]");
    if (M >= ((int64_t)1 << 31) - 1 || (int64_t)n * k >= ((int64_t)1 << 31))
        return fail(BP_ERR_UNSUPPORTED, "graph too large for 32-bit device indexing");
    if (!row_ptr || (M > 0 && (!col || !rev)))
        return fail(BP_ERR_INVALID_ARG, "NULL graph array");
    if (row_ptr[0] != 0 || row_ptr[n] != M)
        return fail(BP_ERR_BAD_GRAPH, "row_ptr must start at 0 and end at n_dir_edges");
    std::vector<int32_t> src((size_t)M);
    for (int32_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i] || row_ptr[i + 1] > M)
            return fail(BP_ERR_BAD_GRAPH, "row_ptr not monotone at vertex " + std::to_string(i));
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            src[(size_t)e] = i;
    }
    for (int64_t e = 0; e < M; ++e) {
        int32_t j = col[e], r = rev[e];
        if (j < 0 || j >= n)
            return fail(BP_ERR_BAD_GRAPH, "col out of range at edge " + std::to_string(e));
        if (j == src[(size_t)e])
            return fail(BP_ERR_BAD_GRAPH, "self-loop at edge " + std::to_string(e));
        if (r < 0 || r >= M || r == e)
            return fail(BP_ERR_BAD_GRAPH, "rev out of range at edge " + std::to_string(e));
        if (rev[r] != e)
            return fail(BP_ERR_BAD_GRAPH, "rev is not an involution at edge " + std::to_string(e));
        if (col[r] != src[(size_t)e] || src[(size_t)r] != j)
            return fail(BP_ERR_BAD_GRAPH, "rev[e] is not the opposite edge at edge " + std::to_string(e));
    }
    std::vector<int32_t> gv((size_t)n_graphs + 1), ge((size_t)n_graphs + 1), gid((size_t)std::max(n, 1));
    if (gvo) {
        if (gvo[0] != 0 || gvo[n_graphs] != n)
            return fail(BP_ERR_BAD_GRAPH, "graph_var_offsets must start at 0 and end at n_vars");
        for (int32_t q = 0; q < n_graphs; ++q)
            if (gvo[q + 1] < gvo[q])
                return fail(BP_ERR_BAD_GRAPH, "graph_var_offsets not monotone");
        for (int32_t q = 0; q <= n_graphs; ++q)
            gv[(size_t)q] = (int32_t)gvo[q];
    } else {
        gv[0] = 0;
        gv[1] = n;
    }
    for (int32_t q = 0; q <= n_graphs; ++q)
        ge[(size_t)q] = (int32_t)row_ptr[gv[(size_t)q]];
    for (int32_t q = 0; q < n_graphs; ++q) {
        for (int32_t i = gv[(size_t)q]; i < gv[(size_t)q + 1]; ++i) {
            gid[(size_t)i] = q;
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                if (col[e] < gv[(size_t)q] || col[e] >= gv[(size_t)q + 1])
                    return fail(BP_ERR_BAD_GRAPH, "edge " + std::to_string(e) + " leaves graph " +
                                                      std::to_string(q));
        }
    }
    // Everything above is host-side validation; device work starts here.
    cudaGetDevice(&g->dev);
    prepare_select_kernels();
    prepare_potts_tc();
    prepare_stream_kernels();
    g->n = n;
    g->k = k;
    g->M = M;
    g->G = n_graphs;
    // lanes per vertex of the k-state kernels; above 32 a warp per vertex with
    // 2 (k <= 64) or 4 (k <= 128) states per lane
    g->kp = k <= 4 ? 4 : (k <= 8 ? 8 : (k <= 16 ? 16 : (k <= 32 ? 32 : (k <= 64 ? 64 : 128))));
    g->h_rev.assign(rev, rev + M);
    g->h_col.assign(col, col + M);
    g->h_src = src;
    g->h_gv_off = gv;
    g->h_ge_off = ge;
    int64_t max_keys = 1;
    for (int32_t q = 0; q < n_graphs; ++q) {
        g->max_graph_vertices = std::max(g->max_graph_vertices, gv[(size_t)q + 1] - gv[(size_t)q]);
        g->max_graph_edges = std::max(g->max_graph_edges, ge[(size_t)q + 1] - ge[(size_t)q]);
    }
    for (int32_t q = 0; q < n_graphs; ++q)
        max_keys = std::max<int64_t>(max_keys, std::max<int64_t>(ge[(size_t)q + 1] - ge[(size_t)q],
                                                                 gv[(size_t)q + 1] - gv[(size_t)q]));
    g->sel_smem_bytes = (int32_t)std::min<int64_t>(max_keys * 8, select_smem_limit());
    std::vector<int32_t> rp32((size_t)n + 1);
    for (int32_t i = 0; i <= n; ++i)
        rp32[(size_t)i] = (int32_t)row_ptr[i];
    for (int32_t i = 0; i < n; ++i)
        g->max_deg = std::max<int32_t>(g->max_deg, (int32_t)(row_ptr[i + 1] - row_ptr[i]));
    int rc;
    if ((rc = dalloc(&g->d_row_ptr, (size_t)n + 1 + PAD)) || (rc = dalloc(&g->d_col, (size_t)M)) ||
        (rc = dalloc(&g->d_rev, (size_t)M + PAD)) || (rc = dalloc(&g->d_gid, (size_t)std::max(n, 1))) ||
        (rc = dalloc(&g->d_gv_off, (size_t)n_graphs + 1)) || (rc = dalloc(&g->d_ge_off, (size_t)n_graphs + 1)))
        return rc;
    BP_CK(cudaMemcpy(g->d_row_ptr, rp32.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice));
    if (M) {
        BP_CK(cudaMemcpy(g->d_col, col, sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice));
        BP_CK(cudaMemcpy(g->d_rev, rev, sizeof(int32_t) * (size_t)M, cudaMemcpyHostToDevice));
    }
    BP_CK(cudaMemcpy(g->d_gid, gid.data(), sizeof(int32_t) * gid.size(), cudaMemcpyHostToDevice));
    BP_CK(cudaMemcpy(g->d_gv_off, gv.data(), sizeof(int32_t) * gv.size(), cudaMemcpyHostToDevice));
    BP_CK(cudaMemcpy(g->d_ge_off, ge.data(), sizeof(int32_t) * ge.size(), cudaMemcpyHostToDevice));
    // per-graph state, reductions, beliefs
    if ((rc = dalloc(&g->d_gs, (size_t)n_graphs)) || (rc = dalloc(&g->d_red_max, (size_t)n_graphs * NSUB)) ||
        (rc = dalloc(&g->d_red_cnt, (size_t)n_graphs * NSUB)) ||
        (rc = dalloc(&g->d_red_commit, (size_t)n_graphs * NSUB)) ||
        (rc = dalloc(&g->d_red_commit_lo, (size_t)n_graphs * NSUB)) || (rc = dalloc(&g->d_running, 1)) ||
        (rc = dalloc(&g->d_queue, 1)) ||
        (rc = dalloc(&g->d_level, (size_t)std::max(n, 1))) ||
        (rc = dalloc(&g->d_beliefs, (size_t)n * (size_t)k)))
        return rc;
    {
        // tensor-core tiles: greedy runs of vertices, at most 128 edges and 32 vertices
        std::vector<int32_t> tv;
        tv.push_back(0);
        bool ok = true;
        int32_t cur_v = 0;
        int64_t cur_e = 0;
        for (int32_t i = 0; i < n; ++i) {
            const int64_t d = row_ptr[i + 1] - row_ptr[i];
            if (d > 128)
                ok = false;
            if (cur_v > 0 && (cur_v + 1 > 32 || cur_e + d > 128)) {
                tv.push_back(i);
                cur_v = 0;
                cur_e = 0;
            }
            ++cur_v;
            cur_e += d;
        }
        if (n > 0)
            tv.push_back(n);
        g->tc_tiles_ok = ok;
        g->n_tc_tiles = (int32_t)tv.size() - 1;
        if ((rc = dalloc(&g->d_tc_tiles, tv.size())))
            return rc;
        BP_CK(cudaMemcpy(g->d_tc_tiles, tv.data(), sizeof(int32_t) * tv.size(), cudaMemcpyHostToDevice));
        if (ok && g->n_tc_tiles > 0) {
            std::vector<TcTileRec> rec((size_t)g->n_tc_tiles);
            for (int32_t t = 0; t < g->n_tc_tiles; ++t) {
                TcTileRec &r = rec[(size_t)t];
                memset(&r, 0, sizeof(r));
                const int32_t va = tv[(size_t)t], vb = tv[(size_t)t + 1];
                r.va = va;
                r.nvt = vb - va;
                r.e0 = (int32_t)row_ptr[va];
                r.ne = (int32_t)(row_ptr[vb] - row_ptr[va]);
                r.gg0 = gid[(size_t)va];
                r.gg1 = gid[(size_t)vb - 1];
                for (int32_t v = va; v < vb; ++v) {
                    r.rpl[v - va] = (uint8_t)(row_ptr[v] - r.e0);
                    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                        r.src[e - r.e0] = (uint8_t)(v - va);
                        r.rev[e - r.e0] = rev[e];
                    }
                }
                r.rpl[r.nvt] = (uint8_t)r.ne;
            }
            if ((rc = dalloc(&g->d_tc_rec, rec.size())))
                return rc;
            BP_CK(cudaMemcpy(g->d_tc_rec, rec.data(), sizeof(TcTileRec) * rec.size(), cudaMemcpyHostToDevice));
        }
    }
    if ((rc = dalloc(&g->d_err, 1)))
        return rc;
    BP_CK(cudaMemset(g->d_err, 0, sizeof(int32_t)));
    {
        // warp tiles of the streamed update: greedy runs of consecutive
        // vertices of one graph, at most STREAM_WT out-edges and STREAM_WV
        // vertices
        std::vector<int4> rec;
        bool ok = g->max_deg <= STREAM_WT;
        for (int32_t q = 0; ok && q < n_graphs; ++q) {
            int32_t v = gv[(size_t)q];
            const int32_t vend = gv[(size_t)q + 1];
            while (v < vend) {
                const int32_t v0 = v;
                int64_t ecount = 0;
                while (v < vend && v - v0 < STREAM_WV && ecount + (row_ptr[v + 1] - row_ptr[v]) <= STREAM_WT) {
                    ecount += row_ptr[v + 1] - row_ptr[v];
                    ++v;
                }
                // {first vertex, first edge, graph, vertex count}: every
                // vertex lies in one tile, so a tile ends where the next begins
                rec.push_back(make_int4(v0, (int32_t)row_ptr[v0], q, v - v0));
            }
        }
        if (!ok)
            rec.clear();
        g->wtiles_ok = ok;
        g->n_wtiles = (int32_t)rec.size();
        rec.push_back(make_int4(n, (int32_t)M, -1, 0));
        if ((rc = dalloc(&g->d_wtiles, rec.size())))
            return rc;
        BP_CK(cudaMemcpy(g->d_wtiles, rec.data(), sizeof(int4) * rec.size(), cudaMemcpyHostToDevice));
        std::vector<int4> crec;
        for (size_t t = 0; t + 1 < rec.size(); ++t)
            crec.push_back(make_int4(rec[t].y, rec[t + 1].y, rec[t].z, ge[(size_t)rec[t].z]));
        if (!crec.empty()) {
            if ((rc = dalloc(&g->d_ctiles, crec.size())))
                return rc;
            BP_CK(cudaMemcpy(g->d_ctiles, crec.data(), sizeof(int4) * crec.size(), cudaMemcpyHostToDevice));
        }
    }
    BP_CK(cudaMallocHost((void **)&g->h_running, sizeof(int32_t)));
    BP_CK(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    BP_CK(cudaEventCreate(&g->ev0));
    BP_CK(cudaEventCreate(&g->ev1));
    BP_CK(cudaEventCreate(&g->ev_pt0));
    BP_CK(cudaEventCreate(&g->ev_pt1));
    return BP_OK;
}

int create_common(int32_t n_graphs, const int64_t *gvo, int32_t n, int32_t k, int64_t M, const int64_t *row_ptr,
                  const int32_t *col, const int32_t *rev, bp_graph **out)
{
    if (!out)
        return fail(BP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    bp_graph *g = new (std::nothrow) bp_graph();
    if (!g)
        return fail(BP_ERR_OOM, "host allocation failed");
    int rc = validate_and_upload(g, n_graphs, gvo, n, k, M, row_ptr, col, rev);
    if (rc != BP_OK) {
        std::string keep = g_last_error;
        bp_destroy_graph(g);
        g_last_error = keep;
        return rc;
    }
    *out = g;
    return BP_OK;
}

// Update mode of a round: LBP, RnBP with the commit inside the streamed
// update, or candidates and residuals.
int eval_mode(const RunParams &rp)
{
    return rp.schedule == SCHED_LBP ? MODE_LBP : (rp.fused_rnbp ? MODE_RNBP_FUSED : MODE_CAND);
}

// Records one round (evaluation, decision, frontier work) on stream s and
// returns the number of kernels it launched. ev (nullable) receives 5 events:
// round start, after evaluation, after decision, after selection (and splash
// levels), round end (after the splash sweep).
int64_t record_round(bp_graph *g, int dtype, const DevGraph &dg, const DevRun &dr, const RunParams &rp,
                     cudaStream_t s, cudaEvent_t *ev)
{
    const bool any = dg.n > 0;
    int64_t kernels = 0;
    if (ev)
        cudaEventRecord(ev[0], s);
    const int emode = eval_mode(rp);
    if (rp.tc_path)
        launch_potts_tc(dtype, dg, dr, rp, emode, g->d_tc_tiles, g->d_tc_rec, g->n_tc_tiles, rp.tc_path, g->d_err,
                        s);
    else
        launch_eval(dtype, dg, dr, rp, emode, 0, g->kp, s);
    kernels += any;
    if (ev)
        cudaEventRecord(ev[1], s);
    launch_decide(dg, dr, rp, s);
    kernels += 1;
    if (ev)
        cudaEventRecord(ev[2], s);
    switch (rp.schedule) {
    case SCHED_LBP:
        break;
    case SCHED_RNBP:
        if (!rp.fused_rnbp) {
            launch_commit_rnbp(dtype, dg, dr, rp, s);
            kernels += any;
        }
        break;
    case SCHED_RBP:
        launch_select_rbp(dtype, dg, dr, rp, s);
        kernels += (dg.sel_grid[0] && dr.gsel) ? grid_select_launches(dtype, false) : 1;
        break;
    default: {   // SCHED_RS
        launch_select_rs(dtype, dg, dr, rp, s);
        kernels += (dg.sel_grid[1] && dr.gsel) ? grid_select_launches(dtype, true) : 1;
        const int h = rp.splash_depth;
        auto level_of = [h](int step) { return step <= h ? h - step : step - h; };
        // the cluster selection forms the BFS levels (and the level lists) itself
        const bool in_select = !(dg.sel_grid[1] && dr.gsel);
        if (dg.epm == 1 && dr.lvl_list && h <= LVL_MAX) {
            // sweeps over per-level vertex lists
            if (!in_select) {
                for (int d = 1; d < h; ++d)
                    launch_bfs_level(dg, dr, d, s);
                launch_bfs_level_lists(dg, dr, h, h, s);
                kernels += any ? (h > 0 ? h : 1) : 0;
            }
            if (ev)
                cudaEventRecord(ev[3], s);
            auto step_launch = launch_splash_list_step;
            // sweep steps launch without programmatic serialization (measured
            // slower between sweep steps); the next round's update still
            // overlaps the last one, which lets its dependents launch early
            step_launch(dtype, dg, dr, -1, level_of(0), s, false);
            for (int step = 0; step < 2 * h; ++step)
                step_launch(dtype, dg, dr, level_of(step), level_of(step + 1), s, false);
            step_launch(dtype, dg, dr, level_of(2 * h), -1, s, false);
            kernels += any ? 2 * h + 2 : 0;
            break;
        }
        if (!in_select) {
            for (int d = 1; d <= h; ++d)
                launch_bfs_level(dg, dr, d, s);
            kernels += any ? h : 0;
        }
        if (ev)
            cudaEventRecord(ev[3], s);
        if (dg.epm == 1) {
            // binary messages: each sub-step's commit fused with the next evaluation
            launch_splash_step(dtype, dg, dr, -1, level_of(0), s);
            for (int step = 0; step < 2 * h; ++step)
                launch_splash_step(dtype, dg, dr, level_of(step), level_of(step + 1), s);
            launch_splash_step(dtype, dg, dr, level_of(2 * h), -1, s);
            kernels += any ? 2 * h + 2 : 0;
        } else {
            for (int step = 0; step <= 2 * h; ++step) {
                const int L = level_of(step);
                launch_eval(dtype, dg, dr, rp, MODE_SPLASH, L, g->kp, s);
                launch_splash_commit(dtype, dg, dr, L, s);
                kernels += any ? 2 : 0;
            }
        }
    }
    }
    if (ev) {
        if (rp.schedule != SCHED_RS)
            cudaEventRecord(ev[3], s);
        cudaEventRecord(ev[4], s);
    }
    return kernels;
}

// Returns the instantiated graph of `rounds` rounds for these parameters,
// capturing it on first use.
int get_graph_exec(bp_graph *g, int dtype, const RunParams &rp, int rounds, CachedGraph **out)
{
    for (auto &c : g->cache) {
        if (c.dtype == dtype && c.rounds == rounds && c.kp == g->kp && c.epm == epm_of(g) &&
            memcmp(&c.rp, &rp, sizeof(rp)) == 0) {
            *out = &c;
            return BP_OK;
        }
    }
    if (g->cache.size() >= 24) {
        destroy_cached(g->cache.front());
        g->cache.erase(g->cache.begin());
    }
    CachedGraph c;
    c.rp = rp;
    c.dtype = dtype;
    c.rounds = rounds;
    c.kp = g->kp;
    c.epm = epm_of(g);
    c.kernels = 0;
    DevGraph dg = dev_graph(g, dtype);
    apply_select_plan(g, dtype, rp.sel_grid, dg);
    DevRun dr = dev_run(g);
    BP_CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < rounds; ++r)
        c.kernels += record_round(g, dtype, dg, dr, rp, g->cap_stream, nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate");
    g->cache.push_back(c);
    *out = &g->cache.back();
    return BP_OK;
}

// Smallest float whose value is >= x (x > 0, finite).
float float_at_least(double x)
{
    float f = (float)x;
    if ((double)f < x)
        f = std::nextafter(f, std::numeric_limits<float>::infinity());
    return f;
}

bool all_finite(const float *p, size_t n)
{
    for (size_t q = 0; q < n; ++q)
        if (!std::isfinite(p[q]))
            return false;
    return true;
}

// Finite or -inf (an absent state, or an impossible state pair) everywhere.
bool finite_or_neg_inf(const float *p, size_t n)
{
    for (size_t q = 0; q < n; ++q)
        if (!std::isfinite(p[q]) && !(std::isinf(p[q]) && p[q] < 0.0f))
            return false;
    return true;
}

}  // namespace

// Run parameters of (schedule, parallelism, eps, max_rounds, opt) on handle g
// with message storage dtype; variant receives the resolved update mapping.
static int build_run_params(const bp_graph *g, int32_t schedule, double parallelism, double eps, int32_t max_rounds,
                     const bp_options &opt, int dtype, RunParams &rp, int32_t &variant)
{
    memset(&rp, 0, sizeof(rp));
    rp.schedule = schedule;
    rp.max_rounds = max_rounds;
    rp.eps = eps;
    rp.low_p = schedule == BP_LBP ? 1.0 : parallelism;
    rp.high_p = opt.high_p;
    rp.ratio_threshold = opt.ratio_threshold;
    rp.seed = opt.seed;
    rp.graph_id_base = opt.graph_id_base;
    rp.pdl = opt.overlap_launches == 2 ? 0 : 1;
    rp.splash_depth = opt.splash_depth;
    rp.rs_roots_mode = opt.rs_roots_mode;
    rp.dynamic_p = (opt.dynamic_p && (schedule == BP_RBP || schedule == BP_RS)) ? 1 : 0;
    rp.record_trace = (opt.record_trace && opt.trace_capacity > 0 && schedule != BP_LBP) ? 1 : 0;
    rp.trace_capacity = rp.record_trace ? opt.trace_capacity : 0;
    const int64_t trace_count = schedule == BP_RS ? g->n : g->M;
    rp.trace_words = (int32_t)((trace_count + 31) / 32);
    variant = epm_of(g) == 1 ? resolve_variant(g, schedule, dtype, opt.kernel_variant) : 1;
    if (variant == 6 && (dtype == DT_F64 || !g->wtiles_ok))
        return fail(BP_ERR_UNSUPPORTED, "the streamed update (kernel_variant 6) needs FP32, BF16 or Q16 messages "
                                        "and vertices with at most 128 out-edges");
    rp.variant = variant == 3 ? 1 : variant;
    // RnBP on the streamed update: the update commits itself, writing both
    // EdgeRatio outcomes (three message buffers); with a recorded trace the
    // commit kernel runs instead and the update hands it the eps test as flag
    // words
    rp.fused_rnbp = (schedule == BP_RNBP && rp.variant == 6 && !rp.record_trace) ? 1 : 0;
    rp.eps_words = (schedule == BP_RNBP && rp.variant == 6 && !rp.fused_rnbp) ? 1 : 0;
    rp.eps_f = float_at_least(eps);
    // shared-table update in vertex tiles: 0 = per-vertex k-state kernel,
    // 1 = tiles on CUDA cores, 2 = tiles on tensor cores, 3 = tensor cores split
    rp.tc_path = 0;
    if (g->pair_kind == BP_PAIR_SHARED && g->tc_tiles_ok && g->k <= 32 && (dtype == BP_F32 || dtype == BP_BF16)) {
        if (opt.potts_path >= 1)
            rp.tc_path = opt.potts_path;
        else if (g->k >= 16)
            rp.tc_path = 3;
    }
    if (opt.potts_path >= 1 && rp.tc_path == 0)
        return fail(BP_ERR_UNSUPPORTED, "the tiled shared-table update needs a shared table with at most 32 "
                                        "states, FP32/BF16 storage and vertices with at most 128 out-edges");
    return BP_OK;
}

// =========================================================================
extern "C" {

void bp_default_options(bp_options *opt)
{
    if (!opt)
        return;
    memset(opt, 0, sizeof(*opt));
    opt->seed = 0;
    opt->high_p = 1.0;
    opt->ratio_threshold = 0.9;
    opt->splash_depth = 2;
    opt->rs_roots_mode = 0;
    opt->msg_dtype = BP_F32;
    opt->record_trace = 0;
    opt->trace_capacity = 0;
    opt->rounds_per_launch = 0;
    opt->cuda_stream = nullptr;
    opt->time_budget_ms = 0.0;
    opt->graph_id_base = 0;
    opt->kernel_variant = 0;
    opt->profile = 0;
    opt->potts_path = 0;
    opt->select_path = 0;
}

int bp_create_graph(int32_t n_vars, int32_t n_states, int64_t n_dir_edges, const int64_t *row_ptr,
                    const int32_t *col, const int32_t *rev, bp_graph **out)
{
    return create_common(1, nullptr, n_vars, n_states, n_dir_edges, row_ptr, col, rev, out);
}

int bp_create_batch(int32_t n_graphs, const int64_t *graph_var_offsets, int32_t n_states, int64_t n_dir_edges,
                    const int64_t *row_ptr, const int32_t *col, const int32_t *rev, bp_graph **out)
{
    if (n_graphs < 1 || !graph_var_offsets)
        return fail(BP_ERR_INVALID_ARG, "n_graphs < 1 or graph_var_offsets NULL");
    int32_t n = (int32_t)graph_var_offsets[n_graphs];
    if (graph_var_offsets[n_graphs] < 0 || graph_var_offsets[n_graphs] >= ((int64_t)1 << 31))
        return fail(BP_ERR_INVALID_ARG, "bad vertex count");
    return create_common(n_graphs, graph_var_offsets, n, n_states, n_dir_edges, row_ptr, col, rev, out);
}

// Binary Ising potentials: the raw unary log-potentials and couplings are
// copied to the device, where kernels check them and derive the arrays of the
// update (launch_pot_ising), instead of host loops over every edge. The
// buffers keep their addresses across calls (their sizes are fixed by the
// graph), so captured rounds are dropped only when the storage scales change.
static int set_ising_potentials(bp_graph *g, const float *unary_log, const float *beta)
{
    const int32_t n = g->n;
    const int64_t M = g->M;
    int rc;
    g->has_pot = false;
    g->has_result = false;
    if (g->pot_bufs_kind != BP_PAIR_ISING_BETA) {
        dfree(g->d_unary);
        dfree(g->d_udiff32);
        dfree(g->d_udiff64);
        dfree(g->d_q32);
        dfree(g->d_q64);
        dfree(g->d_pair);
        dfree(g->d_psi_shared);
        dfree(g->d_kpresent);
        clear_cache(g);
        g->pot_bufs_kind = -1;
        if ((rc = dalloc(&g->d_unary, (size_t)n * 2)) || (rc = dalloc(&g->d_udiff64, (size_t)n)) ||
            (rc = dalloc(&g->d_udiff32, (size_t)n + PAD)) || (rc = dalloc(&g->d_q64, (size_t)M)) ||
            (rc = dalloc(&g->d_q32, (size_t)M + PAD)))
            return rc;
        g->pot_bufs_kind = BP_PAIR_ISING_BETA;
    }
    if (!g->d_potcheck && (rc = dalloc(&g->d_potcheck, 1)))
        return rc;
    if (n)
        BP_CK(cudaMemcpy(g->d_unary, unary_log, sizeof(float) * (size_t)n * 2, cudaMemcpyHostToDevice));
    if (M)
        BP_CK(cudaMemcpy(g->d_q32, beta, sizeof(float) * (size_t)M, cudaMemcpyHostToDevice));
    PotCheck hc;
    BP_CK(launch_pot_ising(g->d_unary, g->d_q32, g->d_q64, g->d_udiff32, g->d_udiff64, g->d_rev, n, (int)M,
                           g->d_potcheck, &hc));
    if (hc.flags & 1u)
        return fail(BP_ERR_NONFINITE, "NaN or +inf unary log-potential");
    if (hc.flags & 2u)
        return fail(BP_ERR_NONFINITE, "a vertex has no present state");
    if (hc.flags & 4u)
        return fail(BP_ERR_UNSUPPORTED, "absent states (unary -inf) need per-edge tables (BP_PAIR_TABLE)");
    if (hc.flags & 8u)
        return fail(BP_ERR_NONFINITE, "NaN, +inf or (outside tables) -inf pairwise log-potential");
    if (hc.flags & 16u)
        return fail(BP_ERR_NONFINITE, "beta[rev[e]] != beta[e] at edge " + std::to_string(hc.bad_edge));
    float bmaxf;
    memcpy(&bmaxf, &hc.bmax_bits, sizeof(float));
    const double bmax = (double)bmaxf;
    const float qs = bmax > 0.0 ? (float)(2.0 * bmax / 32767.0) : 1.0f / 32767.0f;
    const float bs = bf16_scale(bmax > 0.0 ? bmax : 0.5);
    if (qs != g->qscale || bs != g->bscale)
        clear_cache(g);   // captured rounds hold the storage scales by value
    g->qscale = qs;
    g->bscale = bs;
    g->pair_kind = BP_PAIR_ISING_BETA;
    g->has_pot = true;
    return BP_OK;
}

int bp_set_potentials(bp_graph *g, const float *unary_log, int32_t pair_kind, const float *pair_log)
{
    if (!g || !unary_log || (!pair_log && !(pair_kind == BP_PAIR_ISING_BETA && g->M == 0) &&
                             !(pair_kind == BP_PAIR_TABLE && g->M == 0)))
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    BP_CK(cudaSetDevice(g->dev));
    const int32_t n = g->n, k = g->k;
    const int64_t M = g->M;
    if (pair_kind < 0 || pair_kind > 2)
        return fail(BP_ERR_INVALID_ARG, "unknown pair kind");
    if (pair_kind == BP_PAIR_ISING_BETA && k != 2)
        return fail(BP_ERR_INVALID_ARG, "Ising beta potentials need n_states = 2");
    if (pair_kind == BP_PAIR_ISING_BETA)
        return set_ising_potentials(g, unary_log, pair_log);
    if (!finite_or_neg_inf(unary_log, (size_t)n * k))
        return fail(BP_ERR_NONFINITE, "NaN or +inf unary log-potential");
    // a state with unary log-potential -inf is absent (variable state counts)
    std::vector<int32_t> kpresent((size_t)n, k);
    bool absent = false;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t x = 0; x < k; ++x)
            if (std::isinf(unary_log[(size_t)i * k + x])) {
                --kpresent[(size_t)i];
                absent = true;
            }
        if (kpresent[(size_t)i] == 0)
            return fail(BP_ERR_NONFINITE, "vertex " + std::to_string(i) + " has no present state");
    }
    if (absent && pair_kind != BP_PAIR_TABLE)
        return fail(BP_ERR_UNSUPPORTED, "absent states (unary -inf) need per-edge tables (BP_PAIR_TABLE)");
    // (binary Ising potentials took the device path above)
    size_t plen = pair_kind == BP_PAIR_TABLE ? (size_t)M * k * k : (size_t)k * k;
    if (plen && !(pair_kind == BP_PAIR_TABLE ? finite_or_neg_inf(pair_log, plen) : all_finite(pair_log, plen)))
        return fail(BP_ERR_NONFINITE, "NaN, +inf or (outside tables) -inf pairwise log-potential");
    if (pair_kind == BP_PAIR_TABLE) {
        for (int64_t e = 0; e < M; ++e) {
            const float *a = pair_log + (size_t)e * k * k;
            const float *b = pair_log + (size_t)g->h_rev[(size_t)e] * k * k;
            for (int x = 0; x < k; ++x)
                for (int y = 0; y < k; ++y)
                    if (a[x * k + y] != b[y * k + x])
                        return fail(BP_ERR_NONFINITE, "table(rev[e]) is not table(e) transposed at edge " +
                                                          std::to_string(e));
        }
    } else {
        for (int x = 0; x < k; ++x)
            for (int y = 0; y < k; ++y)
                if (pair_log[x * k + y] != pair_log[y * k + x])
                    return fail(BP_ERR_NONFINITE, "shared pairwise table is not symmetric");
    }
    g->has_pot = false;
    g->has_result = false;
    g->pot_bufs_kind = -1;
    dfree(g->d_unary);
    dfree(g->d_udiff32);
    dfree(g->d_udiff64);
    dfree(g->d_q32);
    dfree(g->d_q64);
    dfree(g->d_pair);
    dfree(g->d_psi_shared);
    dfree(g->d_kpresent);
    clear_cache(g);
    int rc;
    if (absent) {
        if ((rc = dalloc(&g->d_kpresent, (size_t)n)))
            return rc;
        BP_CK(cudaMemcpy(g->d_kpresent, kpresent.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
    }
    if ((rc = dalloc(&g->d_unary, (size_t)n * k)))
        return rc;
    BP_CK(cudaMemcpy(g->d_unary, unary_log, sizeof(float) * (size_t)n * k, cudaMemcpyHostToDevice));
    std::vector<double> ud((size_t)n);
    std::vector<float> ud32((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        ud[(size_t)i] = (double)unary_log[(size_t)i * k + 1] - (double)unary_log[(size_t)i * k];
        ud32[(size_t)i] = (float)ud[(size_t)i];
    }
    if ((rc = dalloc(&g->d_udiff64, (size_t)n)) || (rc = dalloc(&g->d_udiff32, (size_t)n + PAD)))
        return rc;
    if (n) {
        BP_CK(cudaMemcpy(g->d_udiff64, ud.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
        BP_CK(cudaMemcpy(g->d_udiff32, ud32.data(), sizeof(float) * (size_t)n, cudaMemcpyHostToDevice));
    }
    g->qscale = 1.0f / 32767.0f;
    g->bscale = bf16_scale(0.5);
    if (pair_kind == BP_PAIR_TABLE) {
        if ((rc = dalloc(&g->d_pair, plen)))
            return rc;
        if (plen && absent) {
            // no mass on an absent state: a pair involving one is impossible
            // (log-potential -inf), so a message into vertex j is a
            // distribution over j's present states; table(rev e) stays the
            // transpose of table(e)
            std::vector<float> tab(pair_log, pair_log + plen);
            const float ninf = -std::numeric_limits<float>::infinity();
            for (int64_t e = 0; e < M; ++e) {
                const float *ui = unary_log + (size_t)g->h_src[(size_t)e] * k;
                const float *uj = unary_log + (size_t)g->h_col[(size_t)e] * k;
                float *t = tab.data() + (size_t)e * k * k;
                for (int32_t x = 0; x < k; ++x)
                    for (int32_t y = 0; y < k; ++y)
                        if (std::isinf(ui[x]) || std::isinf(uj[y]))
                            t[x * k + y] = ninf;
            }
            BP_CK(cudaMemcpy(g->d_pair, tab.data(), sizeof(float) * plen, cudaMemcpyHostToDevice));
        } else if (plen) {
            BP_CK(cudaMemcpy(g->d_pair, pair_log, sizeof(float) * plen, cudaMemcpyHostToDevice));
        }
    } else {
        if ((rc = dalloc(&g->d_pair, plen)) || (rc = dalloc(&g->d_psi_shared, plen)))
            return rc;
        float mx = pair_log[0];
        for (size_t q = 1; q < plen; ++q)
            mx = std::max(mx, pair_log[q]);
        std::vector<float> psi(plen);
        for (size_t q = 0; q < plen; ++q)
            psi[q] = (float)std::exp((double)pair_log[q] - (double)mx);
        BP_CK(cudaMemcpy(g->d_pair, pair_log, sizeof(float) * plen, cudaMemcpyHostToDevice));
        BP_CK(cudaMemcpy(g->d_psi_shared, psi.data(), sizeof(float) * plen, cudaMemcpyHostToDevice));
    }
    g->pair_kind = pair_kind;
    g->has_pot = true;
    return BP_OK;
}

int bp_run(bp_graph *g, int32_t schedule, double parallelism, double eps, int32_t max_rounds,
           const bp_options *opt_in, bp_run_stats *stats)
{
    if (!g)
        return fail(BP_ERR_INVALID_ARG, "NULL handle");
    if (!g->has_pot)
        return fail(BP_ERR_NO_POTENTIALS, "bp_set_potentials has not been called");
    if (schedule < 0 || schedule > 3)
        return fail(BP_ERR_INVALID_ARG, "unknown schedule");
    if (!(eps > 0.0) || !std::isfinite(eps))
        return fail(BP_ERR_INVALID_ARG, "eps must be positive and finite");
    if (max_rounds < 0)
        return fail(BP_ERR_INVALID_ARG, "max_rounds must be >= 0");
    if (schedule != BP_LBP && (!(parallelism > 0.0) || !std::isfinite(parallelism)))
        return fail(BP_ERR_INVALID_ARG, "parallelism must be positive and finite");
    bp_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        bp_default_options(&opt);
    if (opt.msg_dtype < 0 || opt.msg_dtype > 3)
        return fail(BP_ERR_INVALID_ARG, "unknown msg_dtype");
    if (opt.msg_dtype == BP_Q16 && epm_of(g) != 1)
        return fail(BP_ERR_UNSUPPORTED, "Q16 storage needs the binary Ising layout");
    if (!(opt.high_p >= 0.0) || !std::isfinite(opt.high_p) || !std::isfinite(opt.ratio_threshold))
        return fail(BP_ERR_INVALID_ARG, "bad high_p or ratio_threshold");
    if (opt.potts_path < 0 || opt.potts_path > 3)
        return fail(BP_ERR_INVALID_ARG, "potts_path must be 0..3");
    if (opt.select_path < 0 || opt.select_path > 2)
        return fail(BP_ERR_INVALID_ARG, "select_path must be 0..2");
    if (opt.splash_sweep < 0 || opt.splash_sweep > 1)
        return fail(BP_ERR_INVALID_ARG, "splash_sweep must be 0 or 1");
    if (opt.overlap_launches < 0 || opt.overlap_launches > 2)
        return fail(BP_ERR_INVALID_ARG, "overlap_launches must be 0..2");
    if (opt.dynamic_p < 0 || opt.dynamic_p > 1)
        return fail(BP_ERR_INVALID_ARG, "dynamic_p must be 0 or 1");
    if (opt.dynamic_p && (schedule == BP_RBP || schedule == BP_RS) && !(opt.high_p > 0.0))
        return fail(BP_ERR_INVALID_ARG, "dynamic_p needs high_p > 0 (the RBP / RS HighP fraction)");
    if (opt.kernel_variant < 0 || opt.kernel_variant > 6 || opt.kernel_variant == 2 || opt.kernel_variant == 5)
        return fail(BP_ERR_INVALID_ARG, "kernel_variant must be 0, 1, 3, 4 or 6");
    if (opt.splash_depth < 0 || opt.splash_depth > 16)
        return fail(BP_ERR_INVALID_ARG, "splash_depth must be in [0, 16]");
    if (opt.record_trace && opt.trace_capacity < 0)
        return fail(BP_ERR_INVALID_ARG, "negative trace_capacity");
    BP_CK(cudaSetDevice(g->dev));
    const int dtype = opt.msg_dtype;
    int rc = ensure_msg_buffers(g, dtype);
    if (rc != BP_OK)
        return rc;
    if (schedule == BP_RS && epm_of(g) == 1 && opt.splash_depth <= LVL_MAX && !g->d_lvl_list) {
        // level lists of the Residual Splash sweeps, kept until the handle is destroyed
        if ((rc = dalloc(&g->d_lvl_list, (size_t)(LVL_MAX + 1) * (size_t)std::max(g->n, 1))) != BP_OK ||
            (rc = dalloc(&g->d_lvl_cnt, (size_t)(LVL_MAX + 1))) != BP_OK)
            return rc;
        BP_CK(cudaMemset(g->d_lvl_cnt, 0, sizeof(int32_t) * (LVL_MAX + 1)));
    }

    RunParams rp;
    int32_t variant = 1;
    if ((rc = build_run_params(g, schedule, parallelism, eps, max_rounds, opt, dtype, rp, variant)) != BP_OK)
        return rc;
    if (rp.fused_rnbp && !g->d_msg[2]) {
        // (+ PAD elements like the other two)
        clear_cache(g);
        if ((rc = dalloc((char **)&g->d_msg[2], ((size_t)g->M * (size_t)g->buf_epm + PAD) * dtype_size(dtype))) !=
            BP_OK)
            return rc;
    }
    if (rp.eps_words && !g->d_eps_words) {
        // kept until the handle is destroyed (4 words per warp tile)
        if ((rc = dalloc(&g->d_eps_words, (size_t)g->n_wtiles * 4)) != BP_OK)
            return rc;
    }
    if (rp.record_trace) {
        size_t words = (size_t)rp.trace_capacity * (size_t)rp.trace_words;
        if (words > g->trace_alloc_words) {
            clear_cache(g);
            dfree(g->d_trace);
            if ((rc = dalloc(&g->d_trace, words)) != BP_OK)
                return rc;
            g->trace_alloc_words = words;
        }
    }

    cudaStream_t s = (cudaStream_t)opt.cuda_stream;
    if ((schedule == BP_RBP || schedule == BP_RS) &&
        (!g->sel_planned[dtype] || (resolve_select_path(g, schedule, dtype, opt.select_path) == 2 && !g->d_gsel))) {
        int32_t c[2], dyn[2], grid[2];
        plan_select(dtype, g->G, g->max_graph_edges, g->max_graph_vertices, c, dyn, grid);
        if ((grid[0] || grid[1] || resolve_select_path(g, schedule, dtype, opt.select_path) == 2) &&
            !g->d_gsel) {
            // buffers of the grid-wide selection, kept until the handle is destroyed
            std::vector<int32_t> co(2 * ((size_t)g->G + 1));
            g->n_chunks_rbp = grid_select_chunks(g->h_ge_off.data(), g->G, co.data());
            g->n_chunks_rs = grid_select_chunks(g->h_gv_off.data(), g->G, co.data() + g->G + 1);
            const size_t bins = (size_t)g->G * grid_select_bins();
            if ((rc = dalloc(&g->d_gsel, (size_t)g->G)) != BP_OK ||
                (rc = dalloc(&g->d_gsel_hist, bins)) != BP_OK ||
                (rc = dalloc(&g->d_gsel_tie, (size_t)std::max(g->n_chunks_rbp, g->n_chunks_rs))) != BP_OK ||
                (rc = dalloc(&g->d_chunk_off, co.size())) != BP_OK)
                return rc;
            BP_CK(cudaMemset(g->d_gsel_hist, 0, sizeof(unsigned int) * bins));
            BP_CK(cudaMemcpy(g->d_chunk_off, co.data(), sizeof(int32_t) * co.size(), cudaMemcpyHostToDevice));
            clear_cache(g);   // captured rounds hold the run buffers
        }
        g->sel_plan[dtype][0] = c[0];
        g->sel_plan[dtype][1] = dyn[0];
        g->sel_plan[dtype][2] = grid[0];
        g->sel_plan[dtype][3] = c[1];
        g->sel_plan[dtype][4] = dyn[1];
        g->sel_plan[dtype][5] = grid[1];
        g->sel_planned[dtype] = true;
    }
    DevGraph dg = dev_graph(g, dtype);
    {
        const int32_t sp = resolve_select_path(g, schedule, dtype, opt.select_path);
        int bits = g->sel_planned[dtype] ? (g->sel_plan[dtype][2] | (g->sel_plan[dtype][5] << 1)) : 0;
        if (sp != 0)
            bits = sp == 2 ? 3 : 0;
        if (!g->d_gsel)
            bits = 0;
        apply_select_plan(g, dtype, bits, dg);
        rp.sel_grid = bits;
    }
    DevRun dr = dev_run(g);
    g->has_result = false;
    auto t_start = std::chrono::steady_clock::now();
    int64_t kernels = 0;
    BP_CK(cudaEventRecord(g->ev0, s));
    launch_init(dtype, dg, dr, s);
    kernels += ((size_t)g->M * g->k > 0) + 1;
    BP_CK(cudaMemsetAsync(g->d_err, 0, sizeof(int32_t), s));
    if (rp.record_trace)
        BP_CK(cudaMemsetAsync(g->d_trace, 0, sizeof(uint32_t) * (size_t)rp.trace_capacity * rp.trace_words, s));
    BP_CK(cudaGetLastError());

    // The persistent batch kernel (one cluster per graph, all rounds inside one
    // launch) is taken on request; the automatic choice replays captured rounds,
    // which measured faster on every workload here (the per-round kernels keep
    // 64 warps per SM over the whole batch, a cluster only 32 per SM).
    const bool persistent = epm_of(g) == 1 && variant == 3;
    float batch_ms = 0.f;
    bool stopped = false;
    std::vector<float> t_eval, t_decide, t_front, t_sweep;   // per global round (profile)
    if (persistent) {
        const long long budget_ns = opt.time_budget_ms > 0.0 ? (long long)(opt.time_budget_ms * 1e6) : 0;
        BP_CK(cudaEventRecord(g->ev_pt0, s));
        BP_CK(launch_persistent(dtype, dg, dr, rp, budget_ns, s));
        BP_CK(cudaEventRecord(g->ev_pt1, s));
        kernels += 1;
    } else {
        const int max_chunk = opt.rounds_per_launch > 0 ? opt.rounds_per_launch
                              : (schedule == BP_RS ? 16 : 64);
        int chunk = opt.rounds_per_launch > 0 ? opt.rounds_per_launch : 2;
        int64_t rounds_launched = 0;
        // Each replay runs `chunk` rounds (evaluations); graphs that finish turn the
        // rest of their kernels into no-ops. The host polls the running count once
        // per replay. Automatic chunks double up to max_chunk and never run past
        // the max_rounds + 1 evaluations a graph can need.
        for (;;) {
            if (opt.rounds_per_launch <= 0)
                chunk = (int)std::max<int64_t>(1, std::min<int64_t>(chunk, (int64_t)max_rounds + 1 - rounds_launched));
            if (opt.profile) {
                // direct launches with events between the phases of every round
                if (g->prof_events.size() < (size_t)chunk * 5) {
                    size_t old = g->prof_events.size();
                    g->prof_events.resize((size_t)chunk * 5);
                    for (size_t q = old; q < g->prof_events.size(); ++q)
                        BP_CK(cudaEventCreate(&g->prof_events[q]));
                }
                for (int r = 0; r < chunk; ++r)
                    kernels += record_round(g, dtype, dg, dr, rp, s, &g->prof_events[(size_t)r * 5]);
                BP_CK(cudaGetLastError());
            } else {
                CachedGraph *cg = nullptr;
                if ((rc = get_graph_exec(g, dtype, rp, chunk, &cg)) != BP_OK)
                    return rc;
                BP_CK(cudaGraphLaunch(cg->exec, s));
                kernels += cg->kernels;
            }
            rounds_launched += chunk;
            BP_CK(cudaMemcpyAsync(g->h_running, g->d_running, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            BP_CK(cudaStreamSynchronize(s));
            if (opt.profile) {
                for (int r = 0; r < chunk; ++r) {
                    float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
                    cudaEvent_t *ev = &g->prof_events[(size_t)r * 5];
                    BP_CK(cudaEventElapsedTime(&a, ev[0], ev[1]));
                    BP_CK(cudaEventElapsedTime(&b, ev[1], ev[2]));
                    BP_CK(cudaEventElapsedTime(&c, ev[2], ev[3]));
                    BP_CK(cudaEventElapsedTime(&d, ev[3], ev[4]));
                    t_eval.push_back(a);
                    t_decide.push_back(b);
                    t_front.push_back(c);
                    t_sweep.push_back(d);
                }
            }
            if (*g->h_running <= 0)
                break;
            if (rounds_launched > (int64_t)max_rounds + 1) {
                // cannot happen: every running graph stops after max_rounds + 1 evaluations
                return fail(BP_ERR_CUDA, "round loop did not terminate");
            }
            if (opt.time_budget_ms > 0.0) {
                double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
                if (el > opt.time_budget_ms) {
                    launch_stop_running(dg, dr, s);
                    stopped = true;
                    break;
                }
            }
            chunk = std::min(chunk * 2, max_chunk);
        }
    }
    if (stopped)
        kernels += 1;
    launch_beliefs(dtype, dg, dr, g->kp, s);
    kernels += g->n > 0;
    BP_CK(cudaGetLastError());
    BP_CK(cudaEventRecord(g->ev1, s));
    std::vector<GState> hs((size_t)g->G);
    BP_CK(cudaMemcpyAsync(hs.data(), g->d_gs, sizeof(GState) * (size_t)g->G, cudaMemcpyDeviceToHost, s));
    BP_CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    BP_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    {
        int32_t h_err = 0;
        BP_CK(cudaMemcpy(&h_err, g->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (h_err)
            return fail(BP_ERR_CUDA, "a bulk-copy or tensor-core completion wait expired; results are invalid");
    }
    if (persistent) {
        BP_CK(cudaEventElapsedTime(&batch_ms, g->ev_pt0, g->ev_pt1));
        for (const GState &st : hs)
            stopped = stopped || st.status == ST_STOPPED;
    }

    g->last_stats.assign((size_t)g->G, bp_run_stats());
    bp_run_stats tot;
    memset(&tot, 0, sizeof(tot));
    tot.converged = 1;
    tot.n_graphs = g->G;
    tot.device_ms = ms;
    int32_t max_r = 0;
    bp_profile prof;
    memset(&prof, 0, sizeof(prof));
    prof.kernel_launches = kernels;
    prof.batch_kernel_ms = batch_ms;
    for (int32_t q = 0; q < g->G; ++q) {
        prof.full_evals += (int64_t)hs[(size_t)q].full_evals;
        prof.active_vertices += (int64_t)hs[(size_t)q].full_nodes;
        const GState &st = hs[(size_t)q];
        bp_run_stats &o = g->last_stats[(size_t)q];
        memset(&o, 0, sizeof(o));
        o.converged = st.status == ST_CONVERGED;
        o.rounds = st.rounds;
        o.committed_updates = (int64_t)st.committed;
        o.candidate_evals = (int64_t)st.evals;
        o.final_max_residual = st.final_maxr;
        o.final_unconverged = (int64_t)st.final_cnt;
        o.status = st.status == ST_STOPPED ? BP_ERR_TIMEOUT : BP_OK;
        o.n_graphs = 1;
        o.device_ms = ms;
        tot.converged &= o.converged;
        tot.rounds = std::max(tot.rounds, o.rounds);
        tot.committed_updates += o.committed_updates;
        tot.candidate_evals += o.candidate_evals;
        tot.final_max_residual = std::max(tot.final_max_residual, o.final_max_residual);
        tot.final_unconverged += o.final_unconverged;
        if (o.status != BP_OK)
            tot.status = o.status;
        max_r = std::max(max_r, st.rounds);
    }
    if (opt.profile) {
        // rounds with a running graph: every graph evaluates rounds + 1 times
        const size_t live = std::min(t_eval.size(), (size_t)max_r + 1);
        for (size_t r = 0; r < live; ++r) {
            prof.eval_ms += t_eval[r];
            prof.decide_ms += t_decide[r];
            prof.select_ms += t_front[r];
            prof.sweep_ms += t_sweep[r];
        }
        prof.frontier_ms = prof.select_ms + prof.sweep_ms;
        prof.eval_launches = (int64_t)live;
        // every committing round of an RS run sweeps 2h + 2 fused steps (binary)
        if (schedule == BP_RS && epm_of(g) == 1)
            prof.sweep_launches = (int64_t)(live > 0 ? live - 1 : 0) * (2 * opt.splash_depth + 2);
    }
    for (int w = 0; w < 2; ++w)
        prof.select_ctas[w] = (dg.sel_grid[w] && dr.gsel) ? 0 : dg.sel_c[w];
    prof.kernel_variant = variant;
    prof.sweep_ctas = 0;
    prof.sweep_form = 0;
    prof.overlap_launches = rp.pdl;
    prof.fused_commit = rp.fused_rnbp;
    g->last_profile = prof;
    g->has_result = true;
    g->res_dtype = dtype;
    g->res_schedule = schedule;
    g->trace_rounds = rp.record_trace ? std::min(max_r, rp.trace_capacity) : 0;
    g->trace_words = rp.trace_words;
    if (stats)
        *stats = tot;
    if (stopped)
        return fail(BP_ERR_TIMEOUT, "wall-clock budget ran out; results are from the last committed state");
    return BP_OK;
}

int bp_get_beliefs(const bp_graph *g, double *out)
{
    if (!g || !out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (!g->has_result)
        return fail(BP_ERR_NO_RESULT, "no bp_run result");
    BP_CK(cudaSetDevice(g->dev));
    BP_CK(cudaMemcpy(out, g->d_beliefs, sizeof(double) * (size_t)g->n * g->k, cudaMemcpyDeviceToHost));
    return BP_OK;
}

int bp_get_messages(const bp_graph *g, double *out)
{
    if (!g || !out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (!g->has_result)
        return fail(BP_ERR_NO_RESULT, "no bp_run result");
    BP_CK(cudaSetDevice(g->dev));
    size_t count = (size_t)g->M * g->k;
    if (!count)
        return BP_OK;
    double *d = nullptr;
    int rc = dalloc(&d, count);
    if (rc)
        return rc;
    launch_messages(g->res_dtype, dev_graph(g, g->res_dtype), dev_run(g), g->kp, d, 0);
    cudaError_t e = cudaMemcpy(out, d, sizeof(double) * count, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy messages");
    return BP_OK;
}

int bp_get_residuals(const bp_graph *g, double *out)
{
    if (!g || !out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (!g->has_result)
        return fail(BP_ERR_NO_RESULT, "no bp_run result");
    if (g->res_schedule == BP_LBP)
        return fail(BP_ERR_UNSUPPORTED, "LBP runs keep no residuals");
    if (!g->M)
        return BP_OK;
    BP_CK(cudaSetDevice(g->dev));
    const size_t M = (size_t)g->M;
    if (g->res_dtype == DT_F64) {
        BP_CK(cudaMemcpy(out, g->d_resid, sizeof(double) * M, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp(M);
        BP_CK(cudaMemcpy(tmp.data(), g->d_resid, sizeof(float) * M, cudaMemcpyDeviceToHost));
        for (size_t e = 0; e < M; ++e)
            out[e] = (double)tmp[e];
    }
    return BP_OK;
}

int bp_get_graph_stats(const bp_graph *g, bp_run_stats *out)
{
    if (!g || !out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (!g->has_result)
        return fail(BP_ERR_NO_RESULT, "no bp_run result");
    memcpy(out, g->last_stats.data(), sizeof(bp_run_stats) * g->last_stats.size());
    return BP_OK;
}

int bp_get_trace(const bp_graph *g, uint32_t *out, int64_t capacity_words, int32_t *rounds_out)
{
    if (!g || !rounds_out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (!g->has_result)
        return fail(BP_ERR_NO_RESULT, "no bp_run result");
    *rounds_out = g->trace_rounds;
    size_t words = (size_t)g->trace_rounds * (size_t)g->trace_words;
    if (!words)
        return BP_OK;
    if (!out || capacity_words < (int64_t)words)
        return fail(BP_ERR_INVALID_ARG, "trace buffer too small");
    BP_CK(cudaSetDevice(g->dev));
    BP_CK(cudaMemcpy(out, g->d_trace, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost));
    return BP_OK;
}

int bp_set_graph_parallelism(bp_graph *g, const double *p)
{
    if (!g)
        return fail(BP_ERR_INVALID_ARG, "NULL handle");
    if (!p) {
        if (g->graph_p_set)
            clear_cache(g);   // captured rounds hold the per-graph array
        g->graph_p_set = false;
        return BP_OK;
    }
    for (int32_t q = 0; q < g->G; ++q)
        if (!(p[q] > 0.0) || !std::isfinite(p[q]))
            return fail(BP_ERR_INVALID_ARG, "parallelism of graph " + std::to_string(q) +
                                                " must be positive and finite");
    BP_CK(cudaSetDevice(g->dev));
    int rc;
    if (!g->d_graph_p && (rc = dalloc(&g->d_graph_p, (size_t)g->G)) != BP_OK)
        return rc;
    BP_CK(cudaMemcpy(g->d_graph_p, p, sizeof(double) * (size_t)g->G, cudaMemcpyHostToDevice));
    if (!g->graph_p_set)
        clear_cache(g);
    g->graph_p_set = true;
    return BP_OK;
}

int bp_autotune(bp_graph *g, int32_t schedule, double parallelism, double eps, const bp_options *opt,
                int32_t trial_rounds, bp_tune_result *out)
{
    if (!g || !out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (trial_rounds < 1)
        return fail(BP_ERR_INVALID_ARG, "trial_rounds must be >= 1");
    if (!g->has_pot)
        return fail(BP_ERR_NO_POTENTIALS, "bp_set_potentials has not been called");
    if (epm_of(g) != 1)
        return fail(BP_ERR_UNSUPPORTED, "mapping autotuning covers the binary Ising update");
    bp_options o;
    if (opt)
        o = *opt;
    else
        bp_default_options(&o);
    o.profile = 0;
    o.time_budget_ms = 0.0;
    o.record_trace = 0;
    memset(out, 0, sizeof(*out));
    static const int32_t cand[] = {1, 4, 6, 3};
    double best = std::numeric_limits<double>::infinity();
    int32_t best_v = 1;
    for (int c = 0; c < 4; ++c) {
        if (cand[c] == 3 && g->G == 1)
            continue;   // the persistent kernel runs one cluster per graph
        if (cand[c] == 6 && (o.msg_dtype == BP_F64 || !g->wtiles_ok))
            continue;   // the streamed tiles need FP32 arithmetic and <= 128 out-edges per vertex
        o.kernel_variant = cand[c];
        bp_run_stats st;
        int rc = bp_run(g, schedule, parallelism, eps, trial_rounds, &o, &st);   // warm-up: captures rounds
        if (rc != BP_OK)
            return rc;
        if ((rc = bp_run(g, schedule, parallelism, eps, trial_rounds, &o, &st)) != BP_OK)
            return rc;
        const double ms = st.device_ms / (double)std::max(st.rounds, 1);
        out->ms_per_round[cand[c]] = ms;
        if (ms < best) {
            best = ms;
            best_v = cand[c];
        }
    }
    // RBP and RS: the selection path (cluster kernels or grid-wide kernels)
    // with the chosen mapping
    int32_t best_sp = 0;
    if (schedule == BP_RBP || schedule == BP_RS) {
        double best_s = std::numeric_limits<double>::infinity();
        o.kernel_variant = best_v;
        for (int32_t sp = 1; sp <= 2; ++sp) {
            o.select_path = sp;
            bp_run_stats st;
            int rc = bp_run(g, schedule, parallelism, eps, trial_rounds, &o, &st);
            if (rc != BP_OK)
                return rc;
            if ((rc = bp_run(g, schedule, parallelism, eps, trial_rounds, &o, &st)) != BP_OK)
                return rc;
            const double ms = st.device_ms / (double)std::max(st.rounds, 1);
            out->ms_per_round_select[sp] = ms;
            if (ms < best_s) {
                best_s = ms;
                best_sp = sp;
            }
        }
    }
    const uint32_t key = size_class(g, schedule, o.msg_dtype);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_table[key] = best_v | (best_sp << 8);
    }
    out->kernel_variant = best_v;
    out->select_path = best_sp;
    out->size_class = (int32_t)key;
    g->has_result = false;   // the trial runs leave no result to read
    return BP_OK;
}

int bp_autotune_parallelism(bp_graph *g, int32_t schedule, const double *candidates, int32_t n_candidates,
                            double eps, int32_t max_rounds, const bp_options *opt, double *graph_p_out)
{
    if (!g || !candidates)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (schedule != BP_RNBP && schedule != BP_RBP && schedule != BP_RS)
        return fail(BP_ERR_INVALID_ARG, "parallelism is tuned for RnBP, RBP and RS");
    if (n_candidates < 1 || n_candidates > 64)
        return fail(BP_ERR_INVALID_ARG, "n_candidates must be in [1, 64]");
    for (int32_t c = 0; c < n_candidates; ++c)
        if (!(candidates[c] > 0.0) || !std::isfinite(candidates[c]))
            return fail(BP_ERR_INVALID_ARG, "candidates must be positive and finite");
    int rc;
    if ((rc = bp_set_graph_parallelism(g, nullptr)) != BP_OK)
        return rc;
    // size class of every graph: floor(log2(vertices))
    std::vector<int> cls((size_t)g->G);
    int n_cls = 0;
    for (int32_t q = 0; q < g->G; ++q) {
        cls[(size_t)q] = log2_floor(std::max(1, g->h_gv_off[(size_t)q + 1] - g->h_gv_off[(size_t)q]));
        n_cls = std::max(n_cls, cls[(size_t)q] + 1);
    }
    // score of a candidate on a class: rounds to convergence summed over the
    // class's graphs, a graph that did not converge counting 2 * max_rounds
    std::vector<double> score((size_t)n_cls * (size_t)n_candidates, 0.0);
    std::vector<bp_run_stats> per((size_t)g->G);
    for (int32_t c = 0; c < n_candidates; ++c) {
        if ((rc = bp_run(g, schedule, candidates[c], eps, max_rounds, opt, nullptr)) != BP_OK)
            return rc;
        if ((rc = bp_get_graph_stats(g, per.data())) != BP_OK)
            return rc;
        for (int32_t q = 0; q < g->G; ++q) {
            const bp_run_stats &st = per[(size_t)q];
            score[(size_t)cls[(size_t)q] * n_candidates + c] +=
                st.converged ? (double)st.rounds : 2.0 * (double)max_rounds;
        }
    }
    std::vector<double> chosen((size_t)n_cls, candidates[0]);
    for (int k = 0; k < n_cls; ++k) {
        int best = 0;
        for (int32_t c = 1; c < n_candidates; ++c)
            if (score[(size_t)k * n_candidates + c] < score[(size_t)k * n_candidates + best])
                best = c;
        chosen[(size_t)k] = candidates[best];
    }
    std::vector<double> p((size_t)g->G);
    for (int32_t q = 0; q < g->G; ++q)
        p[(size_t)q] = chosen[(size_t)cls[(size_t)q]];
    if ((rc = bp_set_graph_parallelism(g, p.data())) != BP_OK)
        return rc;
    if (graph_p_out)
        memcpy(graph_p_out, p.data(), sizeof(double) * p.size());
    g->has_result = false;
    return BP_OK;
}

int bp_time_update(bp_graph *g, int32_t schedule, double parallelism, const bp_options *opt_in, int32_t launches,
                   double *ms_per_launch)
{
    if (!g || !ms_per_launch)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (launches < 1)
        return fail(BP_ERR_INVALID_ARG, "launches must be >= 1");
    bp_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        bp_default_options(&opt);
    opt.profile = 0;
    opt.record_trace = 0;
    opt.time_budget_ms = 0.0;
    // a run stopped after its first evaluation sets up every buffer of this
    // configuration (and validates the arguments)
    int rc = bp_run(g, schedule, parallelism, 1e-4, 0, &opt, nullptr);
    if (rc != BP_OK)
        return rc;
    const int dtype = opt.msg_dtype;
    RunParams rp;
    int32_t variant = 1;
    if ((rc = build_run_params(g, schedule, parallelism, 1e-4, 0, opt, dtype, rp, variant)) != BP_OK)
        return rc;
    if (epm_of(g) == 1 && variant == 3)
        return fail(BP_ERR_UNSUPPORTED, "the persistent batch kernel has no separate update launch");
    cudaStream_t s = (cudaStream_t)opt.cuda_stream;
    const DevGraph dg = dev_graph(g, dtype);
    const DevRun dr = dev_run(g);
    const int emode = eval_mode(rp);
    launch_init(dtype, dg, dr, s);
    BP_CK(cudaEventRecord(g->ev0, s));
    for (int32_t l = 0; l < launches; ++l) {
        if (rp.tc_path)
            launch_potts_tc(dtype, dg, dr, rp, emode, g->d_tc_tiles, g->d_tc_rec, g->n_tc_tiles, rp.tc_path, g->d_err,
                        s);
        else
            launch_eval(dtype, dg, dr, rp, emode, 0, g->kp, s);
    }
    BP_CK(cudaEventRecord(g->ev1, s));
    BP_CK(cudaGetLastError());
    BP_CK(cudaEventSynchronize(g->ev1));
    float ms = 0.f;
    BP_CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    *ms_per_launch = (double)ms / launches;
    g->has_result = false;   // the message state is not a run's result
    return BP_OK;
}

int bp_storage_scale(const bp_graph *g, int32_t msg_dtype, float *out)
{
    if (!g || !out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (msg_dtype != BP_Q16 && msg_dtype != BP_BF16)
        return fail(BP_ERR_INVALID_ARG, "msg_dtype must be BP_Q16 or BP_BF16");
    if (!g->has_pot)
        return fail(BP_ERR_NO_POTENTIALS, "bp_storage_scale before bp_set_potentials");
    if (!(g->k == 2 && g->pair_kind == BP_PAIR_ISING_BETA))
        return fail(BP_ERR_UNSUPPORTED, "the scaled 16-bit formats hold binary Ising log-odds");
    *out = storage_scale(g, msg_dtype);
    return BP_OK;
}

int bp_get_profile(const bp_graph *g, bp_profile *out)
{
    if (!g || !out)
        return fail(BP_ERR_INVALID_ARG, "NULL argument");
    if (!g->has_result)
        return fail(BP_ERR_NO_RESULT, "no bp_run result");
    *out = g->last_profile;
    return BP_OK;
}

int bp_graph_info(const bp_graph *g, int32_t *n_vars, int32_t *n_states, int64_t *n_dir_edges, int32_t *n_graphs)
{
    if (!g)
        return fail(BP_ERR_INVALID_ARG, "NULL handle");
    if (n_vars)
        *n_vars = g->n;
    if (n_states)
        *n_states = g->k;
    if (n_dir_edges)
        *n_dir_edges = g->M;
    if (n_graphs)
        *n_graphs = g->G;
    return BP_OK;
}

void bp_destroy_graph(bp_graph *g)
{
    if (!g)
        return;
    cudaSetDevice(g->dev);
    free_run_buffers(g);
    dfree(g->d_row_ptr);
    dfree(g->d_col);
    dfree(g->d_rev);
    dfree(g->d_gid);
    dfree(g->d_gv_off);
    dfree(g->d_ge_off);
    dfree(g->d_unary);
    dfree(g->d_udiff32);
    dfree(g->d_udiff64);
    dfree(g->d_q32);
    dfree(g->d_q64);
    dfree(g->d_pair);
    dfree(g->d_psi_shared);
    dfree(g->d_kpresent);
    dfree(g->d_level);
    dfree(g->d_lvl_list);
    dfree(g->d_lvl_cnt);
    dfree(g->d_graph_p);
    dfree(g->d_gsel);
    dfree(g->d_gsel_hist);
    dfree(g->d_gsel_tie);
    dfree(g->d_chunk_off);
    dfree(g->d_gs);
    dfree(g->d_red_max);
    dfree(g->d_red_cnt);
    dfree(g->d_red_commit);
    dfree(g->d_red_commit_lo);
    dfree(g->d_running);
    dfree(g->d_queue);
    dfree(g->d_tc_tiles);
    dfree(g->d_tc_rec);
    dfree(g->d_err);
    dfree(g->d_potcheck);
    dfree(g->d_wtiles);
    dfree(g->d_ctiles);
    dfree(g->d_eps_words);
    dfree(g->d_trace);
    dfree(g->d_beliefs);
    if (g->h_running)
        cudaFreeHost(g->h_running);
    if (g->cap_stream)
        cudaStreamDestroy(g->cap_stream);
    if (g->ev0)
        cudaEventDestroy(g->ev0);
    if (g->ev1)
        cudaEventDestroy(g->ev1);
    if (g->ev_pt0)
        cudaEventDestroy(g->ev_pt0);
    if (g->ev_pt1)
        cudaEventDestroy(g->ev_pt1);
    for (auto ev : g->prof_events)
        cudaEventDestroy(ev);
    delete g;
}

const char *bp_status_string(int status)
{
    switch (status) {
    case BP_OK: return "ok";
    case BP_ERR_INVALID_ARG: return "invalid argument";
    case BP_ERR_BAD_GRAPH: return "invalid graph";
    case BP_ERR_NO_POTENTIALS: return "potentials not set";
    case BP_ERR_NONFINITE: return "non-finite or inconsistent potentials";
    case BP_ERR_CUDA: return "CUDA error";
    case BP_ERR_TIMEOUT: return "time budget exhausted";
    case BP_ERR_OOM: return "out of memory";
    case BP_ERR_UNSUPPORTED: return "unsupported configuration";
    case BP_ERR_NO_RESULT: return "no result available";
    case BP_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
    }
}

const char *bp_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
