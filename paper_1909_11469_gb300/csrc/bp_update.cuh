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

// Residual Splash sweep step for vertex i with level lv: commit its
// out-messages when lv == Lc, or evaluate them when lv == Le (reading an
// incoming message from buffer 1 when its source is at level Lc). Returns the
// number of messages committed.
template <typename S>
__device__ __forceinline__ unsigned int splash_vertex_bin(const DevGraph &g, const DevRun &dr, int i, int lv,
                                                          int Lc, int Le)
{
    using A = typename Store<S>::A;
    S *b0 = (S *)dr.msg[0];
    S *b1 = (S *)dr.msg[1];
    const int beg = g.row_ptr[i], end = g.row_ptr[i + 1];
    if (Lc >= 0 && lv == Lc) {
        for (int e = beg; e < end; ++e)
            b0[e] = b1[e];
        return (unsigned int)(end - beg);
    }
    if (!(Le >= 0 && lv == Le))
        return 0u;
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
    auto incoming = [&](int e) -> A {
        const int f = g.rev[e];
        const bool fresh = Lc >= 0 && dr.level[g.col[e]] == Lc;
        return Store<S>::ld((fresh ? b1 : b0) + f, g.qscale);
    };
    const int deg = end - beg;
#pragma unroll
    for (int k = 0; k < CACHE; ++k) {
        if (k < deg) {
            uin[k] = incoming(beg + k);
            h += uin[k];
        }
    }
    for (int e = beg + CACHE; e < end; ++e)
        h += incoming(e);
#pragma unroll
    for (int k = 0; k < CACHE; ++k)
        if (k < deg)
            Store<S>::st(b1 + beg + k, ising_logodds(q[beg + k], h - uin[k]), g.qscale);
    for (int e = beg + CACHE; e < end; ++e)
        Store<S>::st(b1 + e, ising_logodds(q[e], h - incoming(e)), g.qscale);
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
