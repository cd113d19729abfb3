// Host-side launchers of the round kernels (internal to libbp_gb300).
#pragma once

#include "bp_internal.cuh"

#include <string>

namespace bpg {

// update modes: LBP (new messages), candidates + residuals (RBP, RnBP, RS),
// Residual Splash sweep evaluation, and the RnBP round with its commit fused
// (the streamed update writes both EdgeRatio outcomes; see bp_stream.cu)
enum { MODE_LBP = 0, MODE_CAND = 1, MODE_SPLASH = 2, MODE_RNBP_FUSED = 3 };
enum { SCHED_LBP = 0, SCHED_RBP = 1, SCHED_RS = 2, SCHED_RNBP = 3 };
enum { DT_F64 = 0, DT_F32 = 1, DT_BF16 = 2, DT_Q16 = 3 };

void launch_init(int dtype, const DevGraph &g, const DevRun &dr, cudaStream_t s);
// Binary Ising potentials on the device (bp_set_potentials): checks, then
// (when every check passes) the derived arrays. beta_q32 holds beta on entry
// and exp(-2 beta) in FP32 on return; host_check receives the checks (flags
// bit 0 unary NaN / +inf, bit 1 a vertex without a present state, bit 2 an
// absent state, bit 3 non-finite beta, bit 4 beta[rev e] != beta[e] with the
// lowest such e in bad_edge) and max |beta| as float bits. Synchronous.
struct PotCheck {
    unsigned flags;
    int bad_edge;
    unsigned bmax_bits;
    int pad;
};
cudaError_t launch_pot_ising(const float *unary, float *beta_q32, double *q64, float *ud32, double *ud64,
                             const int32_t *rev, int n, int M, PotCheck *check, PotCheck *host_check);
void launch_eval(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode, int level_L,
                 int kp, cudaStream_t s);
// Streamed warp-tile update (bp_stream.cu, update mapping 6; FP32, BF16, Q16).
void prepare_stream_kernels();
void launch_eval_stream(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode,
                        cudaStream_t s);
void launch_decide(const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s);
// Loads the kernels of an FP32 thread-per-vertex LBP run (update, decision,
// beliefs) on the current device now rather than at their first launch (the
// runtime loads device code lazily, and a load can allocate device memory).
cudaError_t preload_lbp_f32_kernels();
void launch_commit_rnbp(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s);
// One-time attribute set-up of the selection kernels (dynamic shared memory).
void prepare_select_kernels();
int select_smem_limit();
// Cluster shape of the RBP and RS selection launches for this graph set and
// storage format (host occupancy queries; call outside stream capture).
// grid_out[w] = 1 where the grid-wide kernels are estimated faster (a few large graphs).
void plan_select(int dtype, int G, int max_ge, int max_gv, int32_t c_out[2], int32_t dyn_out[2],
                 int32_t grid_out[2]);
void launch_select_rbp(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s);
void launch_select_rs(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s);
// Grid-wide selection for a few large graphs (bp_select_grid.cu): kernels per
// call, chunk offsets of a graph set (returns the chunk count), histogram bins.
void launch_select_rbp_grid(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s);
void launch_select_rs_grid(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, cudaStream_t s);
int grid_select_launches(int dtype, bool rs);
int grid_select_chunks(const int32_t *off, int G, int32_t *chunk_off);
int grid_select_bins();
void launch_bfs_level(const DevGraph &g, const DevRun &dr, int d, cudaStream_t s);
// Residual Splash (binary messages): commit level Lc and evaluate level Le
// in one kernel (Lc or Le may be -1).
void launch_splash_step(int dtype, const DevGraph &g, const DevRun &dr, int Lc, int Le, cudaStream_t s);
// Residual Splash over per-level vertex lists (binary messages, depth <=
// LVL_MAX): the last BFS level (d = h; d = 0 for depth 0) builds the lists and
// the round's per-graph counts; the list steps pair commits and evaluations
// as launch_splash_step does.
void launch_bfs_level_lists(const DevGraph &g, const DevRun &dr, int d, int h, cudaStream_t s);
// pdl: launch with programmatic stream serialization.
void launch_splash_list_step(int dtype, const DevGraph &g, const DevRun &dr, int Lc, int Le, cudaStream_t s,
                             bool pdl = false);
void launch_splash_commit(int dtype, const DevGraph &g, const DevRun &dr, int level_L, cudaStream_t s);
void launch_stop_running(const DevGraph &g, const DevRun &dr, cudaStream_t s);
void launch_beliefs(int dtype, const DevGraph &g, const DevRun &dr, int kp, cudaStream_t s);
void launch_messages(int dtype, const DevGraph &g, const DevRun &dr, int kp, double *out, cudaStream_t s);

// Persistent batch kernel (binary Ising): every round of every graph in one
// launch, one thread-block cluster per graph at a time.
cudaError_t launch_persistent(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp,
                              long long budget_ns, cudaStream_t s);

// Static description of one shared-table tile (built on the host with the
// tiles): its vertex and edge range, the graphs of its first and last vertex,
// the local first row of every vertex (rpl[nvt] = ne), the local source vertex
// and the rev of every row (0 past the tile). A multiple of 16 bytes.
struct TcTileRec {
    int32_t va, nvt, e0, ne;
    int32_t gg0, gg1, pad0, pad1;
    uint8_t rpl[48];
    uint8_t src[128];
    int32_t rev[128];
};
static_assert(sizeof(TcTileRec) % 16 == 0, "tile records are copied in 16-byte words");

// Shared-table (Potts) update in tiles of consecutive vertices with at most
// 128 out-edges and 32 vertices (tile_v, n_tiles + 1 entries; tile_rec, one
// record per tile); path 1 = CUDA cores, 2 = tensor cores with BF16 products,
// 3 = tensor cores with the BF16 residual products added. FP32 or BF16 storage.
void prepare_potts_tc();
void launch_potts_tc(int dtype, const DevGraph &g, const DevRun &dr, const RunParams &rp, int mode,
                     const int *tile_v, const TcTileRec *tile_rec, int n_tiles, int path, int *err_flag,
                     cudaStream_t s);

// Sets the calling thread's message returned by bp_last_error().
void set_last_error(const std::string &msg);

}  // namespace bpg
