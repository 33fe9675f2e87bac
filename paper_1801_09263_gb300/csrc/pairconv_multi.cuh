// Persistent multi-instance pair-convolution kernel (template), shared by
// the translation units that instantiate it for each block size
// (pairconv_multi*.cu).  See pairconv_multi.cu for the design.
#pragma once

#include <algorithm>
#include <cstring>

#include "grid_sync.cuh"
#include "lace_internal.cuh"
#include "pairconv_generic.cuh"
#include "pairconv_spec2.cuh"

namespace lace {
namespace multi {

constexpr int kMaxEntries = 256;  // instance pieces per chunk

struct ChunkTable {
    int n;                       // entries
    int q[kMaxEntries];          // instance
    int g0[kMaxEntries];         // first grid (instance-local index)
    int cnt[kMaxEntries];        // grids
    size_t pool[kMaxEntries];    // pool offset of the first grid (complex elements)
    size_t ep[kMaxEntries];      // epart offset (doubles)
    int grp[kMaxEntries];        // thread groups a CTA runs at once on the entry's items (1: the whole CTA)
    int item[kMaxEntries + 1];   // prefix of the current phase's work units (one unit = grp items)
    // where the next chunk starts
    int next_q, next_g;
};

// Thread 0: the chunk starting at grid g of instance q.
static __device__ void build_chunk(const MultiArgs& A, int q, int g, ChunkTable& t) {
    size_t pool_used = 0, ep_used = 0;
    int n = 0;
    while (q < A.n_inst && n < kMaxEntries) {
        const int total = A.n_grids[q];
        const int rem = total - g;
        if (rem <= 0) {
            ++q;
            g = 0;
            continue;
        }
        const MultiInst& I = A.inst[q];
        const size_t ng = I.P.ng;
        const size_t per_ep = 2 * (size_t)I.n1;
        const size_t fit_pool = (A.pool_elems - pool_used) / ng;
        const size_t fit_ep = (A.epart_elems - ep_used) / per_ep;
        const int fit = (int)std::min<size_t>((size_t)rem, std::min(fit_pool, fit_ep));
        if (fit <= 0) break;
        t.q[n] = q;
        t.g0[n] = g;
        t.cnt[n] = fit;
        t.pool[n] = pool_used;
        t.ep[n] = ep_used;
        pool_used += (size_t)fit * ng;
        ep_used += (size_t)fit * per_ep;
        ++n;
        g += fit;
        if (g >= total) {
            ++q;
            g = 0;
        }
    }
    t.n = n;
    t.next_q = q;
    t.next_g = g;
}

// Threads of one group for the size-specialised bodies of cubic size n in a
// CTA of nt threads: about one butterfly a thread in the larger radix stage
// of a plane (24: 144 butterflies, 32-48: 256-384, 60 and 64: 600, 512).
__host__ __device__ constexpr int group_threads(int n, int nt) {
    const int g = n <= 24 ? 128 : (n <= 48 ? 256 : 512);
    return g < nt ? g : nt;
}
// Shared memory of one group of size n (16-byte multiple).
__host__ __device__ inline size_t group_smem(int n) { return (spec2::smem_max(n) + 15) / 16 * 16; }
// Groups a CTA of nt threads with smem_cta bytes of dynamic shared memory
// runs at once on items of size n (named barriers 1..15); 0 if none fits.
__host__ __device__ inline int groups_for(int n, int nt, size_t smem_cta) {
    const int by_threads = nt / group_threads(n, nt);
    const int by_smem = (int)(smem_cta / group_smem(n));
    const int g = by_threads < by_smem ? by_threads : by_smem;
    return g < 15 ? g : 15;
}

// Thread 0: unit prefix for a phase (0: planes n1, 1: slabs n2, 2: grids).
// In phases 0 and 1 a unit is grp items of one entry, taken by one CTA at once.
template <int NT, bool SPEC>
static __device__ void build_items(const MultiArgs& A, ChunkTable& t, int phase) {
    int acc = 0;
    for (int e = 0; e < t.n; ++e) {
        t.item[e] = acc;
        const MultiInst& I = A.inst[t.q[e]];
        const int per = phase == 0 ? I.n1 : (phase == 1 ? I.n2 : 1);
        int g = 1;
        if (SPEC && I.spec && phase < 2) {
            g = groups_for(I.spec, NT, A.smem_cta);
            if (g < 1) g = 1;  // the host sizes smem_cta for one group of every size
        }
        t.grp[e] = g;
        acc += (t.cnt[e] * per + g - 1) / g;
    }
    t.item[t.n] = acc;
}

static __device__ __forceinline__ int find_entry(const ChunkTable& t, int it) {
    int lo = 0, hi = t.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.item[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One work unit through the size-specialised pass bodies of
// pairconv_spec2.cuh (the instance's cubic size): the CTA's threads split
// into G groups of group_threads(n, NT), group gi taking item loc0 + gi of
// entry e with its own shared memory, energy scratch and named barrier 1 + gi.
// phase 0: pass A of a plane, 1: pass B of a slab, 2: pass C of a plane (a
// constant at every call site, so each phase loop inlines only its bodies).
// Planes are taken plane-major within each entry (the groups and CTAs in
// flight share the orbital planes of one x).
template <int NT>
__device__ __forceinline__ void spec_unit(int phase, const MultiArgs& A, const ChunkTable& t, int e,
                                          const MultiInst& I, int loc0, unsigned char* smem, double* red) {
    const int G = t.grp[e];
    const int cnt = t.cnt[e];
    const int items = cnt * (phase == 1 ? I.n2 : I.n1);
#define LACE_SPEC_UNIT(NN)                                                                 \
    case NN: {                                                                             \
        constexpr int T = group_threads(NN, NT);                                           \
        const int gi = (int)threadIdx.x / T;                                               \
        const int loc = loc0 + gi;                                                         \
        if (gi < G && loc < items) {                                                       \
            int k, w;                                                                      \
            if (phase == 1) {                                                              \
                k = loc / I.n2;                                                            \
                w = loc - k * I.n2;                                                        \
            } else {                                                                       \
                w = loc / cnt;                                                             \
                k = loc - w * cnt;                                                         \
            }                                                                              \
            spec2::GridView V;                                                             \
            V.psi = I.P.psi;                                                               \
            V.W = I.P.W;                                                                   \
            V.ktab = I.P.ktab;                                                             \
            V.scr = A.pool + t.pool[e] + (size_t)k * I.P.ng;                               \
            V.ep = A.epart + t.ep[e] + (size_t)k * I.n1 * 2;                               \
            V.d = I.P.grids[t.g0[e] + k];                                                  \
            V.n_occ = I.P.n_occ;                                                           \
            V.dv = I.P.dv;                                                                 \
            const spec2::Sub<T> grp{(int)threadIdx.x - gi * T, 1 + gi};                    \
            float4* sm = reinterpret_cast<float4*>(smem + (size_t)gi * group_smem(NN));    \
            if (phase == 0) spec2::body_a<NN, T>(I.P, V, w, sm, nullptr, grp);             \
            else if (phase == 1) spec2::body_b<NN, T>(I.P, V, w, sm, grp);                 \
            else spec2::body_c<NN, T>(I.P, V, w, sm, red + gi * 2 * (T / 32), grp);        \
        }                                                                                  \
    } break;
    switch (I.spec) {
        LACE_SPEC_UNIT(24)
        LACE_SPEC_UNIT(32)
        LACE_SPEC_UNIT(36)
        LACE_SPEC_UNIT(40)
        LACE_SPEC_UNIT(48)
        LACE_SPEC_UNIT(50)
        LACE_SPEC_UNIT(54)
        LACE_SPEC_UNIT(60)
        LACE_SPEC_UNIT(64)
        default: break;
    }
#undef LACE_SPEC_UNIT
}

// SPEC: instances with I.spec run the size-specialised bodies in thread
// groups (spec_unit); the others, and every instance without SPEC, the
// generic-radix bodies on the whole CTA.  Planes are taken plane-major within
// each run of grids of one instance, so the CTAs in flight share the orbital
// planes of one x.
template <int NT, bool SPEC, int MINB = (512 / NT > 0 ? 512 / NT : 1)>
__global__ void __launch_bounds__(NT, MINB) pairconv_multi_kernel(MultiArgs A, int chunk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<float>* work = reinterpret_cast<cplx<float>*>(smem_raw);
    __shared__ ChunkTable t;
    __shared__ double red[2 * 32];
    __shared__ int abort_sh;
    unsigned gen = 0;
    if (threadIdx.x == 0) {
        int q = 0, g = 0;
        for (int c = 0;; ++c) {
            build_chunk(A, q, g, t);
            if (c == chunk || t.n == 0) break;
            q = t.next_q;
            g = t.next_g;
        }
    }
    __syncthreads();
    if (t.n == 0) return;
    // A: planes
    if (threadIdx.x == 0) build_items<NT, SPEC>(A, t, 0);
    __syncthreads();
    for (int u = blockIdx.x; u < t.item[t.n]; u += gridDim.x) {
        const int e = find_entry(t, u);
        const MultiInst& I = A.inst[t.q[e]];
        __syncthreads();  // the previous unit's shared memory is free
        if (SPEC && I.spec) {
            spec_unit<NT>(0, A, t, e, I, (u - t.item[e]) * t.grp[e], smem_raw, red);
        } else {
            const int loc = u - t.item[e], x = loc / t.cnt[e], k = loc - x * t.cnt[e];
            cplx<float>* scr = A.pool + t.pool[e] + (size_t)k * I.P.ng;
            gen::pass_a_plane<float>(I.P, I.P.grids[t.g0[e] + k], scr, x, work);
        }
    }
    if (!grid_barrier(A.bar, gen, &abort_sh)) return;
    // B: slabs
    if (threadIdx.x == 0) build_items<NT, SPEC>(A, t, 1);
    __syncthreads();
    for (int u = blockIdx.x; u < t.item[t.n]; u += gridDim.x) {
        const int e = find_entry(t, u);
        const MultiInst& I = A.inst[t.q[e]];
        __syncthreads();
        if (SPEC && I.spec) {
            spec_unit<NT>(1, A, t, e, I, (u - t.item[e]) * t.grp[e], smem_raw, red);
        } else {
            const int loc = u - t.item[e], k = loc / I.n2, ky = loc - k * I.n2;
            cplx<float>* scr = A.pool + t.pool[e] + (size_t)k * I.P.ng;
            gen::pass_b_slab<float>(I.P, scr, ky, work);
        }
    }
    if (!grid_barrier(A.bar, gen, &abort_sh)) return;
    // C: planes
    if (threadIdx.x == 0) build_items<NT, SPEC>(A, t, 0);
    __syncthreads();
    for (int u = blockIdx.x; u < t.item[t.n]; u += gridDim.x) {
        const int e = find_entry(t, u);
        const MultiInst& I = A.inst[t.q[e]];
        __syncthreads();
        if (SPEC && I.spec) {
            spec_unit<NT>(2, A, t, e, I, (u - t.item[e]) * t.grp[e], smem_raw, red);
        } else {
            const int loc = u - t.item[e], x = loc / t.cnt[e], k = loc - x * t.cnt[e];
            cplx<float>* scr = A.pool + t.pool[e] + (size_t)k * I.P.ng;
            double* ep = A.epart + t.ep[e] + (size_t)k * I.n1 * 2;
            gen::pass_c_plane<float>(I.P, I.P.grids[t.g0[e] + k], scr, x, work, red, ep + (size_t)x * 2);
        }
    }
    if (!grid_barrier(A.bar, gen, &abort_sh)) return;
    // D: per grid, the plane energies in a fixed order -> E[i][j] = E[j][i]
    if (threadIdx.x == 0) build_items<NT, SPEC>(A, t, 2);
    __syncthreads();
    for (int it = blockIdx.x * NT + threadIdx.x; it < t.item[t.n]; it += gridDim.x * NT) {
        const int e = find_entry(t, it);
        const MultiInst& I = A.inst[t.q[e]];
        const int k = it - t.item[e];
        const PairGrid d = I.P.grids[t.g0[e] + k];
        const double* ep = A.epart + t.ep[e] + (size_t)k * I.n1 * 2;
        double sa = 0.0, sb = 0.0;
        for (int x = 0; x < I.n1; ++x) {
            sa += ep[2 * x];
            sb += ep[2 * x + 1];
        }
        const int no = I.P.n_occ;
        if (d.j1 < no) {
            I.E[(size_t)d.i1 * no + d.j1] = sa;
            I.E[(size_t)d.j1 * no + d.i1] = sa;
        }
        if (d.j2 >= 0 && d.j2 < no) {
            I.E[(size_t)d.i2 * no + d.j2] = sb;
            I.E[(size_t)d.j2 * no + d.i2] = sb;
        }
    }
}

}  // namespace multi
}  // namespace lace
