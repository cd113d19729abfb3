// Per-vertex work of the binary Ising update, shared by the per-round kernels
// and the persistent batch kernel so that both compute bit-identical values.
#pragma once

#include "bp_internal.cuh"

namespace bpg {

// Full evaluation of every out-message of vertex i (Eq. 2 in log-odds, Eq. 4
// residual). cur holds the committed messages, out receives the candidates;
// R (MODE_CAND) receives the residuals. maxa / cnt accumulate the largest
// residual and the messages with residual >= eps.
template <typename S, bool STORE_R>
__device__ __forceinline__ void eval_vertex_bin(const DevGraph &g, const S *cur, S *out,
                                                typename ResidT<S>::T *R, int i,
                                                typename Store<S>::A eps_a,
                                                typename Store<S>::A &maxa, unsigned int &cnt)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
    const int deg = end - beg;
    A h;
    const A *q;
    if constexpr (sizeof(A) == 8) {
        h = g.udiff64[i];
        q = (const A *)g.q64;
    } else {
        h = g.udiff32[i];
        q = (const A *)g.q32;
    }
    constexpr int CACHE = 8;
    A uin[CACHE];
#pragma unroll
    for (int c = 0; c < CACHE; ++c) {
        if (c < deg) {
            uin[c] = Store<S>::ld(cur + g.rev[beg + c], g.qscale);
            h += uin[c];
        }
    }
    for (int e = beg + CACHE; e < end; ++e)
        h += Store<S>::ld(cur + g.rev[e], g.qscale);
    auto one = [&](int e, A u_in) {
        const A unew = ising_logodds(q[e], h - u_in);
        const A uq = Store<S>::quant(unew, g.qscale);
        const A r = fabs(m_sigmoid(uq) - m_sigmoid(Store<S>::ld(cur + e, g.qscale)));
        Store<S>::st(out + e, unew, g.qscale);
        if (STORE_R)
            R[e] = (RT)r;
        maxa = r > maxa ? r : maxa;
        cnt += (r >= eps_a) ? 1u : 0u;
    };
#pragma unroll
    for (int c = 0; c < CACHE; ++c)
        if (c < deg)
            one(beg + c, uin[c]);
    for (int e = beg + CACHE; e < end; ++e)
        one(e, Store<S>::ld(cur + g.rev[e], g.qscale));
}

// The same arithmetic as eval_vertex_bin (identical results), with the loads
// arranged for a short dependency chain: the vertex's graph arrays (row range,
// rev, q) are read before the graph's run status is known, so the message
// gathers wait on one level of loads instead of three. gg = graph of vertex i.
// Returns false (and touches nothing) when the graph is not running.
// WAIT: call griddep_wait between the graph arrays (constant during a run)
// and the first read of run state.
template <typename S, bool STORE_R, int CACHE, bool WAIT = false>
__device__ __forceinline__ bool eval_vertex_bin_pf(const DevGraph &g, const DevRun &dr,
                                                   typename ResidT<S>::T *R, int i, int gg,
                                                   typename Store<S>::A eps_a,
                                                   typename Store<S>::A &maxa, unsigned int &cnt)
{
    using A = typename Store<S>::A;
    using RT = typename ResidT<S>::T;
    const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
    const int deg = end - beg;
    A h;
    const A *q;
    if constexpr (sizeof(A) == 8) {
        h = g.udiff64[i];
        q = (const A *)g.q64;
    } else {
        h = g.udiff32[i];
        q = (const A *)g.q32;
    }
    int rv[CACHE];
    A qv[CACHE];
#pragma unroll
    for (int c = 0; c < CACHE; ++c) {
        if (c < deg) {
            rv[c] = g.rev[beg + c];
            qv[c] = q[beg + c];
        }
    }
    if constexpr (WAIT)
        griddep_wait();
    const int status = dr.gs[gg].status;
    const int cb = dr.gs[gg].cur;
    if (status != ST_RUNNING)
        return false;
    const S *cur = (const S *)msg_buf(dr, cb);
    S *out = (S *)msg_buf(dr, cb ^ 1);
    A uin[CACHE], old[CACHE];
#pragma unroll
    for (int c = 0; c < CACHE; ++c) {
        if (c < deg) {
            uin[c] = Store<S>::ld(cur + rv[c], g.qscale);
            old[c] = Store<S>::ld(cur + beg + c, g.qscale);
        }
    }
#pragma unroll
    for (int c = 0; c < CACHE; ++c)
        if (c < deg)
            h += uin[c];
    for (int e = beg + CACHE; e < end; ++e)
        h += Store<S>::ld(cur + g.rev[e], g.qscale);
    auto one = [&](int e, A u_in, A qe, A u_old) {
        const A unew = ising_logodds(qe, h - u_in);
        const A uq = Store<S>::quant(unew, g.qscale);
        const A r = fabs(m_sigmoid(uq) - m_sigmoid(u_old));
        Store<S>::st(out + e, unew, g.qscale);
        if (STORE_R)
            R[e] = (RT)r;
        maxa = r > maxa ? r : maxa;
        cnt += (r >= eps_a) ? 1u : 0u;
    };
#pragma unroll
    for (int c = 0; c < CACHE; ++c)
        if (c < deg)
            one(beg + c, uin[c], qv[c], old[c]);
    for (int e = beg + CACHE; e < end; ++e)
        one(e, Store<S>::ld(cur + g.rev[e], g.qscale), q[e], Store<S>::ld(cur + e, g.qscale));
    return true;
}

// Residual Splash commit of vertex i: its out-messages move from the
// candidate buffer (1) to the state buffer (0). Returns the number committed.
template <typename S>
__device__ __forceinline__ unsigned int splash_commit_vertex(const DevGraph &g, const DevRun &dr, int i)
{
    S *b0 = (S *)dr.msg[0];
    const S *b1 = (const S *)dr.msg[1];
    const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
    for (int e = beg; e < end; ++e)
        b0[e] = b1[e];
    return (unsigned int)(end - beg);
}

// Residual Splash evaluation of vertex i: new out-messages into buffer 1, an
// incoming message read from buffer 1 when its source is at level Lc (written
// by the previous sub-step, committed by this one), else from buffer 0.
template <typename S, int CACHE = 8>
__device__ __forceinline__ void splash_eval_vertex(const DevGraph &g, const DevRun &dr, int i, int Lc)
{
    using A = typename Store<S>::A;
    const S *b0 = (const S *)dr.msg[0];
    S *b1 = (S *)dr.msg[1];
    const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
    A h;
    const A *q;
    if constexpr (sizeof(A) == 8) {
        h = g.udiff64[i];
        q = (const A *)g.q64;
    } else {
        h = g.udiff32[i];
        q = (const A *)g.q32;
    }
    A uin[CACHE];
    auto incoming = [&](int e) -> A {
        const int f = g.rev[e];
        const bool fresh = Lc >= 0 && dr.level[g.col[e]] == Lc;
        return Store<S>::ld((fresh ? (const S *)b1 : b0) + f, g.qscale);
    };
    const int deg = end - beg;
    // the first CACHE incoming messages: both buffers are read next to the
    // source's level, so the value does not wait for the level
    int rf[CACHE], rc[CACHE];
#pragma unroll
    for (int k = 0; k < CACHE; ++k) {
        if (k < deg) {
            rf[k] = g.rev[beg + k];
            rc[k] = g.col[beg + k];
        }
    }
#pragma unroll
    for (int k = 0; k < CACHE; ++k) {
        if (k < deg) {
            const A u0 = Store<S>::ld(b0 + rf[k], g.qscale);
            if (Lc >= 0) {
                const A u1 = Store<S>::ld((const S *)b1 + rf[k], g.qscale);
                uin[k] = dr.level[rc[k]] == Lc ? u1 : u0;
            } else {
                uin[k] = u0;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CACHE; ++k)
        if (k < deg)
            h += uin[k];
    for (int e = beg + CACHE; e < end; ++e)
        h += incoming(e);
#pragma unroll
    for (int k = 0; k < CACHE; ++k)
        if (k < deg)
            Store<S>::st(b1 + beg + k, ising_logodds(q[beg + k], h - uin[k]), g.qscale);
    for (int e = beg + CACHE; e < end; ++e)
        Store<S>::st(b1 + e, ising_logodds(q[e], h - incoming(e)), g.qscale);
}

// The same commit and evaluation for a list entry that carries the vertex's
// first out-edge beg: the first out-edges' graph arrays (and, for the commit,
// the candidates) load next to row_ptr[i + 1] instead of after it. Loads
// past the vertex's last edge stay inside the arrays (index < M) and are not
// used.
template <typename S>
__device__ __forceinline__ unsigned int splash_commit_vertex_b(const DevGraph &g, const DevRun &dr, int i, int beg)
{
    S *b0 = (S *)dr.msg[0];
    const S *b1 = (const S *)dr.msg[1];
    constexpr int CACHE = 4;
    S v[CACHE];
#pragma unroll
    for (int k = 0; k < CACHE; ++k)
        if (beg + k < g.M)
            v[k] = b1[beg + k];
    const int end = g.row_ptr[i + 1];
#pragma unroll
    for (int k = 0; k < CACHE; ++k)
        if (beg + k < end)
            b0[beg + k] = v[k];
    for (int e = beg + CACHE; e < end; ++e)
        b0[e] = b1[e];
    return (unsigned int)(end - beg);
}

template <typename S, int CACHE>
__device__ __forceinline__ void splash_eval_vertex_b(const DevGraph &g, const DevRun &dr, int i, int beg, int Lc)
{
    using A = typename Store<S>::A;
    const S *b0 = (const S *)dr.msg[0];
    S *b1 = (S *)dr.msg[1];
    A h;
    const A *q;
    if constexpr (sizeof(A) == 8) {
        h = g.udiff64[i];
        q = (const A *)g.q64;
    } else {
        h = g.udiff32[i];
        q = (const A *)g.q32;
    }
    int rf[CACHE], rc[CACHE];
#pragma unroll
    for (int k = 0; k < CACHE; ++k) {
        if (beg + k < g.M) {
            rf[k] = g.rev[beg + k];
            rc[k] = g.col[beg + k];
        }
    }
    const int end = g.row_ptr[i + 1];
    const int deg = end - beg;
    // the source's level picks the buffer, so each incoming message is one
    // load (reading both buffers next to the level measured slower: the
    // sweep is bound by its scattered requests more than by their latency)
    A uin[CACHE];
#pragma unroll
    for (int k = 0; k < CACHE; ++k) {
        if (k < deg) {
            const bool fresh = Lc >= 0 && dr.level[rc[k]] == Lc;
            uin[k] = Store<S>::ld((fresh ? (const S *)b1 : b0) + rf[k], g.qscale);
        }
    }
    auto incoming = [&](int e) -> A {
        const int f = g.rev[e];
        const bool fresh = Lc >= 0 && dr.level[g.col[e]] == Lc;
        return Store<S>::ld((fresh ? (const S *)b1 : b0) + f, g.qscale);
    };
#pragma unroll
    for (int k = 0; k < CACHE; ++k)
        if (k < deg)
            h += uin[k];
    for (int e = beg + CACHE; e < end; ++e)
        h += incoming(e);
#pragma unroll
    for (int k = 0; k < CACHE; ++k)
        if (k < deg)
            Store<S>::st(b1 + beg + k, ising_logodds(q[beg + k], h - uin[k]), g.qscale);
    for (int e = beg + CACHE; e < end; ++e)
        Store<S>::st(b1 + e, ising_logodds(q[e], h - incoming(e)), g.qscale);
}

// Residual Splash sweep step for vertex i with level lv: commit its
// out-messages when lv == Lc, or evaluate them when lv == Le. Returns the
// number of messages committed.
template <typename S>
__device__ __forceinline__ unsigned int splash_vertex_bin(const DevGraph &g, const DevRun &dr, int i, int lv,
                                                          int Lc, int Le)
{
    if (Lc >= 0 && lv == Lc)
        return splash_commit_vertex<S>(g, dr, i);
    if (Le >= 0 && lv == Le)
        splash_eval_vertex<S>(g, dr, i, Lc);
    return 0u;
}

// One level of the multi-source splash BFS (pull form): an unreached vertex
// next to a vertex of level d - 1 gets level d.
__device__ __forceinline__ void bfs_vertex(const DevGraph &g, const DevRun &dr, int i, int d)
{
    if (dr.level[i] >= 0)
        return;
    for (int e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
        if (dr.level[g.col[e]] == d - 1) {
            dr.level[i] = (int8_t)d;
            return;
        }
    }
}

}  // namespace bpg
