// The FMM plan behind kifmm_plan: operators, per-target evaluation rows, work lists
// and check-potential buffers for one (tree, kernel, order, precision).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include <memory>

#include "common.cuh"

namespace kifmm {

struct PairTiles {
    DBuf<int4> tiles;               // (op, first pair, pair count, chain flag); count <= the tile cap
    DBuf<int> pin, pout;            // input box, output box per pair
    DBuf<int> kcount;               // mixed M2L with chains: tiles per CTA (else empty)
    std::vector<int> level_tile;    // per level: [level_tile[l], level_tile[l+1]) tiles (U2U/L2L)
    int ntiles = 0;
    int64_t npairs = 0;
};

constexpr int kPairTile = 64;
// events per profiled matvec: 0..8 bound the 8 phases on the matvec's stream (8 = end),
// 9 and 10 bound the near field (on the near-field stream when it overlaps the far field)
constexpr int kPhaseEvents = 11;

// Device scratch of the boundary-integral operators and GMRES, kept between calls
// (the Krylov basis stays resident for the next solve on the same plan).
struct BieScratch {
    DBuf<double> q, krylov, w, r;
};

// Translation tables of one (device, order, cutoffs, precision, ADL centring): shared by
// every plan with that key, freed with the last of them.  FP64 form: m2m/m2l/l2l in
// FP64, Qp x Qp each.  Mixed form: every translation acts between projections onto
// the ranges of the pseudo-inverses (P = W U^T, U orthonormal): families 0 M2M''
// = U_u^T M2M' W_u (Ku x Ku), 1 M2L'' = U_d^T M2L' W_u (Kd x Ku), 2 L2L'' = U_d^T
// L2L' W_d (Kd x Kd), and the projections 3 U_u^T and 4 U_d^T (K x Qp), as FP16 hi/lo
// tables scaled by 2^texp, with their TMA tensor maps.  ru / rd: the ranks, Ku / Kd:
// rounded up to 16.
constexpr int kFamilies = 5;
struct OpTables {
    int device = 0, p = 0;
    double cut_up = 0, cut_dn = 0;  // truncation of Pu and Pd, relative to sigma_max
    int cap_up = 0, cap_dn = 0;     // and at most this many singular triplets (0: no cap)
    bool fp64 = true, centered = false;
    bool cheb = false;              // the Chebyshev engine's tables
    int ru = 0, rd = 0, Ku = 0, Kd = 0;
    int ks = 0;                     // mixed: S2U points (skeleton of the up-check surface)
    DBuf<float> surf_up;            // mixed: those points on the unit surface, ks x 3
    DBuf<double> m2m_d, m2l_d, l2l_d;
    DBuf<__half> tab_h[kFamilies], tab_l[kFamilies];
    int texp[kFamilies] = {0, 0, 0, 0, 0};
    CUtensorMap tmaps[kFamilies][2];
    int64_t bytes() const {
        int64_t b = m2m_d.bytes() + m2l_d.bytes() + l2l_d.bytes() + surf_up.bytes();
        for (int f = 0; f < kFamilies; ++f) b += tab_h[f].bytes() + tab_l[f].bytes();
        return b;
    }
};

struct Plan {
    kifmm_tree_s* tree = nullptr;
    int kernel = 0, p = 0, Q = 0, Qp = 0, prec = 0;
    int nc = 1;                     // output components per target (the field: 3)
    bool cheb = false;              // far field by Chebyshev interpolation (p = nodes per dimension)
    double cut_up = 0, cut_dn = 0;  // pseudo-inverse truncations (up: Pu, down: Pd)
    int cap_up = 0, cap_dn = 0;     // and rank caps (mixed form; 0: none)
    bool fp64 = true;

    // translation tables (shared, see OpTables), each Qp x Qp row-major; D2T rows in
    // the working precision; mixed: bexp the per-box input scales and vin_h/vin_l the
    // scaled, split projected vectors a translation reads (nbox x max(Ku, Kd) each), and
    // sexp, sin_h/sin_l the same for the full check potentials the surface kernels
    // write for the projections (nbox x Qp each).  Kept apart, so the splits of the
    // upward pass survive the X list's surface pass and serve M2L as well.
    std::shared_ptr<OpTables> ops;
    DBuf<double> d2t_d;
    DBuf<float> d2t_f;
    DBuf<int> bexp, sexp;
    DBuf<__half> vin_h, vin_l, sin_h, sin_l;
    DBuf<double> surf_d;            // Q x 3 unit surface
    DBuf<float> surf_f;

    DBuf<double> snrm, tnrm_d;      // sorted normals (DL: sources; ADL: targets)
    DBuf<float> sxf;                // mixed: sorted source coordinates as FP32 hi/lo pairs, 6 x ns SoA
    DBuf<float> txf;                // mixed, targets apart from the sources: the same for them
    DBuf<float4> bcf;               // mixed: per box {centre hi, h}, {centre lo, 0}, {r_upcheck, r_dncheck}
    DBuf<int> bax;                  // mixed DL: per source leaf, the one axis k of its dipoles (0..2), 3
                                    // (none), or 4 + k when its points also lie in one plane normal to k
    DBuf<float> tnrm_f;             // mixed ADL: sorted target normals, FP32 hi (3 rows) and lo (3 rows)

    // work lists
    DBuf<int> s2u_box, s2u_off, s2u_idx;  // S2U: leaf boxes, CSR of source boxes (itself)
    DBuf<int> p2l_box, p2l_off, p2l_idx;  // X list: boxes, CSR of source leaves
    DBuf<int> tleaf, p2p_off, p2p_idx;    // target leaves, CSR of U + W source boxes
    DBuf<int4> p2p_units;                 // mixed: near-field work units (leaf, first range,
                                          // end range, flags: 1 first of its leaf, 2 leaf split)
    DBuf<longlong2> p2p_ranges;           // mixed: source index ranges of the units
    int n_p2p_units = 0, n_p2p_split = 0;
    int64_t near_pairs = 0;               // mixed: (target, source) pairs the near field evaluates
    DBuf<int4> p2p_cunits;                // mixed: one unit per range with close pairs (the
    DBuf<longlong2> p2p_cranges;          //   corrected-distance launch) and those ranges
    int n_p2p_corr = 0;
    int n_p2p_axis = 0;                   // DL: the last units of p2p_units, dipoles along one axis
    int64_t near_axis_pairs = 0;          // their (target, source) pairs
    int64_t near_zero_pairs = 0;          // DL: coplanar pairs dropped (exact zeros)
    bool p2p_multi = false;               // some leaf spans several units
    int n_s2u = 0, n_p2l = 0, n_tleaf = 0;
    int64_t n_xpairs = 0;
    PairTiles u2u, m2l, l2l;
    int64_t m2l_chain_pairs = 0;    // mixed: V pairs in chains (targets written once per chain)
    PairTiles proj_up, proj_x;      // mixed: (box -> box) projections of the S2U leaves'
                                    // up-check and the X-list boxes' down-check potentials
    DBuf<float> zu, zd;             // mixed: projected check potentials, nbox x Ku / Kd
    int max_trg_leaf = 0;
    int tile_cap = kPairTile;       // pairs per translation tile
    DBuf<int> err;                  // device error word (bounded waits that gave up)

    // per-matvec buffers
    DBuf<double> u_d, d_d, res_d, q_d;
    DBuf<float> u_f, d_f, res_f, q_f;

    BieScratch bie;

    // profiling: per-matvec slots of 8 events, reduced when read
    bool profile = false;
    bool serial = false;            // profiling: the near field after the far field, on one stream
    double setup_ms[5] = {};        // set-up phases (ms): tables, work lists, tiles, rows, total
    std::vector<std::vector<cudaEvent_t>> ev_slots;
    int slots_used = 0;
    int launches = 0;
    int64_t device_bytes = 0;

    // captured matvec (kifmm_fmm_matvec_graph): the executable graph, the q / out it
    // was captured for, and the private stream it was captured on
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // mixed: after the gather the far field runs on a highest-priority stream and the
    // near field on a lowest-priority one, so the near field's blocks fill the SMs the
    // far field's many short launches leave idle; both join the caller's stream before
    // the far-field sum is added
    cudaStream_t near_stream = nullptr, far_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_far = nullptr, ev_zero = nullptr;
    const double* g_q = nullptr;
    double* g_out = nullptr;

    // host buffers (kifmm_fmm_matvec_host), set up on first use: inverse permutations
    // (input index -> sorted position) of sources and targets, device staging of a
    // pageable q and of the near sums; while a call runs, io_in (the first kernel reads
    // q in input order and scatters it) and io_out (the last kernel writes f there, in
    // input order); the graph captured for one (q, out) pair of such calls
    DBuf<int64_t> isperm, itperm;
    DBuf<double> q_stage, out_stage;
    bool io_in = false;
    double* io_out = nullptr;
    cudaGraphExec_t hexec = nullptr;
    const double* h_q = nullptr;
    double* h_out = nullptr;
    double* h_io_out = nullptr;

    ~Plan() {
        for (auto& sl : ev_slots)
            for (auto e : sl)
                if (e) cudaEventDestroy(e);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (hexec) cudaGraphExecDestroy(hexec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (ev_far) cudaEventDestroy(ev_far);
        if (ev_zero) cudaEventDestroy(ev_zero);
        if (near_stream) cudaStreamDestroy(near_stream);
        if (far_stream) cudaStreamDestroy(far_stream);
    }
};

}  // namespace kifmm

struct kifmm_plan_s {
    kifmm::Plan P;
};
