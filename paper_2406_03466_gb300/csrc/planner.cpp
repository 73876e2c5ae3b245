// Host planner for the on-chip engine.  See svk_types.h for the program model.
#include "planner.h"

#include <algorithm>
#include <cstring>
#include <unordered_map>

namespace svk {
namespace {

int find_pos(const std::vector<int> &v, int x) {
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i] == x) return (int)i;
    return -1;
}

uint32_t cx_apply(uint32_t v, int c, int t) { return v ^ (((v >> c) & 1u) << t); }

inline uint64_t mix(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h * 0xff51afd7ed558ccdull;
}

uint32_t lop_qubits(const LOp &o) {
    return o.kind == 0 ? (1u << o.a) : ((1u << o.a) | (1u << o.b));
}

}  // namespace

std::string fuse_circuit(const sv_circuit &c, bool fuse, FusedCircuit *F) {
    const int n = c.n_qubits;
    if (n < 1 || n > kNMax) return "n_qubits must be in [1, 30]";
    if (c.n_gates < 0 || (c.n_gates > 0 && !c.gates)) return "circuit has no gate array";
    if (c.n_params < 0 || c.input_dim < 0) return "negative n_params or input_dim";
    *F = FusedCircuit();
    std::vector<std::vector<Member>> gm;  // members per group
    std::vector<int> gq;                  // qubit per group
    std::vector<int> open(n, -1);
    auto close = [&](int q) {
        if (open[q] >= 0) {
            F->lops.push_back({0, q, -1, open[q]});
            open[q] = -1;
        }
    };
    for (int g = 0; g < c.n_gates; ++g) {
        const sv_gate &G = c.gates[g];
        const int t = G.target;
        if (t < 0 || t >= n) return "gate " + std::to_string(g) + ": target out of range";
        Member m{};
        m.param = -1;
        m.angle = 0.0;
        bool single = true;
        switch (G.op) {
        case SV_GATE_RX: m.kind = M_RX; break;
        case SV_GATE_RY: m.kind = M_RY; break;
        case SV_GATE_RZ: m.kind = M_RZ; break;
        case SV_GATE_X: m.kind = M_X; break;
        case SV_GATE_H: m.kind = M_H; break;
        case SV_GATE_ENC_RY_ASIN: m.kind = M_ENC_RY_ASIN; break;
        case SV_GATE_ENC_RZ_ACOS_SQ: m.kind = M_ENC_RZ_ACOS_SQ; break;
        case SV_GATE_CNOT:
        case SV_GATE_CZ: single = false; break;
        default: return "gate " + std::to_string(g) + ": unknown op";
        }
        if (single) {
            if (m.kind <= M_RZ) {
                if (G.param >= c.n_params)
                    return "gate " + std::to_string(g) + ": param index out of range";
                m.param = G.param < 0 ? -1 : G.param;
                m.angle = G.angle;
            } else if (m.kind == M_ENC_RY_ASIN || m.kind == M_ENC_RZ_ACOS_SQ) {
                if (G.param < 0 || G.param >= c.input_dim)
                    return "gate " + std::to_string(g) + ": input column out of range";
                m.param = G.param;
            }
            if (!fuse || open[t] < 0) {
                gm.emplace_back();
                gq.push_back(t);
                open[t] = (int)gm.size() - 1;
            }
            gm[open[t]].push_back(m);
            if (!fuse) close(t);
        } else {
            const int ctl = G.control;
            if (ctl < 0 || ctl >= n || ctl == t)
                return "gate " + std::to_string(g) + ": bad control qubit";
            close(ctl);
            close(t);
            F->lops.push_back({G.op == SV_GATE_CNOT ? 1 : 2, ctl, t, -1});
        }
    }
    for (int q = 0; q < n; ++q) close(q);
    for (size_t g = 0; g < gm.size(); ++g) {
        Group grp{};
        grp.m_begin = (int)F->members.size();
        grp.qubit = gq[g];
        grp.real = 1;
        for (const Member &m : gm[g]) {
            F->members.push_back(m);
            if (m.kind <= M_RZ && m.param >= 0) grp.has_param = 1;
            if (!(m.kind == M_RY || m.kind == M_X || m.kind == M_H || m.kind == M_ENC_RY_ASIN))
                grp.real = 0;
        }
        grp.m_end = (int)F->members.size();
        F->groups.push_back(grp);
    }
    return "";
}

void stage_lops(const std::vector<LOp> &lops, const std::vector<int> &pos, int t, int R, int w,
                HostProgram *P, bool one_per_bit) {
    // lops act on positions pos[qubit] in [0, t); R <= t register bits.
    std::vector<int> Q;
    std::vector<Op> sops;
    std::vector<uint32_t> col(t);
    uint32_t dirty = 0;
    int n_u1 = 0;
    bool any = false;
    const int first_stage = (int)P->stages.size();
    auto reset = [&]() {
        Q.clear();
        sops.clear();
        for (int b = 0; b < t; ++b) col[b] = 1u << b;
        dirty = 0;
        n_u1 = 0;
        any = false;
    };
    auto close_stage = [&]() {
        for (int p = 0; (int)Q.size() < R && p < t; ++p)
            if (find_pos(Q, p) < 0) Q.push_back(p);
        Stage st{};
        bool any_cz = false;
        for (const Op &o : sops) any_cz |= o.kind != OP_U1;
        if (!any_cz) {
            // fused groups on different register bits commute: order by bit
            std::stable_sort(sops.begin(), sops.end(),
                             [](const Op &x, const Op &y) { return x.a < y.a; });
            st.sorted = 1;
            int k = 0;
            for (int i = 0; i <= kRMax; ++i) {
                while (k < (int)sops.size() && sops[k].a < i) ++k;
                st.bit_begin[i] = k;
            }
            st.bit_begin[kRMax] = (int)sops.size();
            // every register bit carries exactly one group, all real: the
            // kernels' straight-line path
            bool one_real = true;
            for (int i = 0; i < R && one_real; ++i)
                one_real = st.bit_begin[i + 1] - st.bit_begin[i] == 1 &&
                           P->groups[(size_t)sops[(size_t)st.bit_begin[i]].group].real;
            if (one_real) st.sorted = 2;
        }
        st.op_begin = (int)P->ops.size();
        for (const Op &o : sops) P->ops.push_back(o);
        st.op_end = (int)P->ops.size();
        st.n_thr = t - R;
        st.n_u1 = n_u1;
        // Thread bit order: the first w thread bits (the lanes of one
        // wavefront) take positions whose swizzled load vectors and store
        // vectors both have independent low w bits, so that those lanes hit
        // distinct banks on the load and on the store; then the rest.
        std::vector<int> rest, order;
        for (int p = 0; p < t; ++p)
            if (find_pos(Q, p) < 0) rest.push_back(p);
        {
            // every subset of min(w, |rest|) positions (at most C(12, 4)):
            // the largest load rank + store rank of the low w bits
            const uint32_t lowm = (1u << w) - 1u;
            auto rank = [&](const uint32_t *v, int m) {
                uint32_t bas[32] = {};
                int r = 0;
                for (int i = 0; i < m; ++i) {
                    uint32_t x = v[i];
                    for (int h = w - 1; h >= 0 && x; --h)
                        if ((x >> h) & 1u) {
                            if (bas[h]) {
                                x ^= bas[h];
                            } else {
                                bas[h] = x;
                                ++r;
                                break;
                            }
                        }
                }
                return r;
            };
            const int m = std::min<int>(w, (int)rest.size()), nr = (int)rest.size();
            uint32_t best_mask = 0;
            int best = -1;
            for (uint32_t sel = 0; sel < (1u << nr); ++sel) {
                if (__builtin_popcount(sel) != m) continue;
                uint32_t vl[32], vs[32];
                int k = 0;
                for (int i = 0; i < nr; ++i)
                    if ((sel >> i) & 1u) {
                        vl[k] = swizzle(1u << rest[i], w) & lowm;
                        vs[k] = swizzle(col[rest[i]], w) & lowm;
                        ++k;
                    }
                const int sc = rank(vl, m) + rank(vs, m);
                if (sc > best) {
                    best = sc;
                    best_mask = sel;
                }
            }
            for (int i = 0; i < nr; ++i)
                if ((best_mask >> i) & 1u) order.push_back(rest[i]);
        }
        for (int p : rest)
            if (find_pos(order, p) < 0) order.push_back(p);
        for (int i = 0; i < kRMax; ++i) {
            st.q[i] = i < R ? Q[i] : -1;
            st.ldq[i] = i < R ? swizzle(1u << Q[i], w) : 0u;
            st.stq[i] = i < R ? swizzle(col[Q[i]], w) : 0u;
        }
        for (int k = 0; k < kNMax; ++k) {
            const bool on = k < t - R;
            st.tpos[k] = on ? order[k] : -1;
            st.ldt[k] = on ? swizzle(1u << order[k], w) : 0u;
            st.stt[k] = on ? swizzle(col[order[k]], w) : 0u;
        }
        P->stages.push_back(st);
        P->perm_cols.push_back(col);
        reset();
    };
    reset();
    for (const LOp &o : lops) {
        if (o.kind == 0) {
            const int q = pos[o.a];
            if (((dirty >> q) & 1u) || n_u1 >= kMaxGroupOpsPerStage) close_stage();
            int idx = find_pos(Q, q);
            if (idx >= 0 && one_per_bit) {
                bool taken = false;
                for (const Op &x : sops) taken |= x.kind == OP_U1 && x.a == idx;
                if (taken) {
                    close_stage();
                    idx = -1;
                }
            }
            if (idx < 0) {
                if ((int)Q.size() >= R) close_stage();
                Q.push_back(q);
                idx = (int)Q.size() - 1;
            }
            sops.push_back({OP_U1, idx, -1, o.group});
            ++n_u1;
            any = true;
        } else if (o.kind == 1) {
            const int a = pos[o.a], b = pos[o.b];
            for (int k = 0; k < t; ++k) col[k] = cx_apply(col[k], a, b);
            dirty |= (1u << a) | (1u << b);
            any = true;
        } else {
            const int a = pos[o.a], b = pos[o.b];
            if (dirty & ((1u << a) | (1u << b))) close_stage();
            sops.push_back({OP_CZ, a, b, -1});
            any = true;
        }
    }
    if (any || (int)P->stages.size() == first_stage) close_stage();
}

void build_thread_bases(HostProgram *P, int t) {
    const int T = 1 << (t - P->R);
    P->tbase.assign((size_t)P->stages.size() * T, ThreadBase{});
    for (size_t s = 0; s < P->stages.size(); ++s) {
        const Stage &st = P->stages[s];
        for (int tid = 0; tid < T; ++tid) {
            ThreadBase b{0u, 0u, 0u, 0u};
            for (int k = 0; k < st.n_thr; ++k)
                if ((tid >> k) & 1) {
                    b.lb ^= st.ldt[k];
                    b.sb ^= st.stt[k];
                    b.lg |= 1u << st.tpos[k];
                }
            P->tbase[s * T + tid] = b;
        }
    }
}

std::string plan_circuit(const sv_circuit &c, int reg_bits, bool fuse, int swz_bits,
                         HostProgram *P) {
    if (reg_bits < 1 || reg_bits > kRMax) return "reg_bits must be in [1, 5]";
    FusedCircuit F;
    std::string err = fuse_circuit(c, fuse, &F);
    if (!err.empty()) return err;
    const int n = c.n_qubits;
    *P = HostProgram();
    P->n = n;
    P->R = std::min(reg_bits, n);
    P->n_params = c.n_params;
    P->input_dim = c.input_dim;
    P->swz_bits = swz_bits;
    P->members = F.members;
    P->groups = F.groups;
    std::vector<int> pos(n);
    for (int q = 0; q < n; ++q) pos[q] = q;
    stage_lops(F.lops, pos, n, P->R, swz_bits, P, false);
    build_thread_bases(P, n);
    return "";
}

std::string plan_passes(const sv_circuit &c0, int tile_bits, int coalesce_bits, int reg_bits,
                        bool fuse, int swz_bits, HostProgram *P, bool relabel) {
    // CZ(a, b) = H_b CNOT(a -> b) H_b: tile passes run fused single-qubit
    // groups and CNOT permutations only.
    std::vector<sv_gate> gates;
    if (c0.n_gates > 0 && c0.gates) {
        for (int g = 0; g < c0.n_gates; ++g) {
            sv_gate G = c0.gates[g];
            if (G.op == SV_GATE_CZ) {
                sv_gate h{};
                h.op = SV_GATE_H;
                h.target = G.target;
                h.control = -1;
                h.param = -1;
                sv_gate cx = G;
                cx.op = SV_GATE_CNOT;
                gates.push_back(h);
                gates.push_back(cx);
                gates.push_back(h);
            } else {
                gates.push_back(G);
            }
        }
    }
    sv_circuit c = c0;
    if (!gates.empty()) {
        c.gates = gates.data();
        c.n_gates = (int)gates.size();
    }
    FusedCircuit F;
    std::string err = fuse_circuit(c, fuse, &F);
    if (!err.empty()) return err;
    const int n = c.n_qubits;
    if (tile_bits < 2 || tile_bits > n || tile_bits > kTileBitsMax) return "tile_bits must be in [2, min(n, 13)]";
    if (coalesce_bits < 0 || coalesce_bits + 2 > tile_bits) return "coalesce_bits too large";
    if (reg_bits < 1 || reg_bits > kRMax || reg_bits > tile_bits) return "bad reg_bits";
    const int t = tile_bits;
    *P = HostProgram();
    P->n = n;
    P->R = reg_bits;
    P->n_params = c.n_params;
    P->input_dim = c.input_dim;
    P->swz_bits = swz_bits;
    P->members = F.members;
    P->groups = F.groups;
    // phys[q]: the bit of the amplitude index that holds qubit q; who[b]: the
    // qubit held by bit b.
    std::vector<int> phys(n), who(n);
    for (int q = 0; q < n; ++q) phys[q] = who[q] = q;
    std::vector<int> pending(F.lops.size());
    for (size_t i = 0; i < pending.size(); ++i) pending[i] = (int)i;
    while (!pending.empty()) {
        uint32_t forced = 0;
        for (int b = 0; b < coalesce_bits; ++b) forced |= 1u << who[b];
        uint32_t L = forced, blocked = 0;
        std::vector<int> taken, rest;
        for (int idx : pending) {
            const uint32_t q = lop_qubits(F.lops[idx]);
            if (q & blocked) {
                blocked |= q;
                rest.push_back(idx);
            } else if ((q & ~L) == 0) {
                taken.push_back(idx);
            } else if (__builtin_popcount(L | q) <= t) {
                L |= q;
                taken.push_back(idx);
            } else {
                blocked |= q;
                rest.push_back(idx);
            }
        }
        if (taken.empty()) return "internal: pass planner made no progress";
        // Spare local qubits: with relabeling, the qubits that the ops left
        // for later passes need first (they can then move to the low bits);
        // otherwise (and then) the lowest qubits.
        if (relabel)
            for (size_t i = 0; i < rest.size() && __builtin_popcount(L) < t; ++i) {
                const uint32_t q = lop_qubits(F.lops[rest[i]]);
                if (__builtin_popcount(L | q) <= t) L |= q;
            }
        for (int p = 0; __builtin_popcount(L) < t && p < n; ++p) L |= 1u << who[p];
        // Tile bit b: the b-th lowest index bit among the local qubits (tile
        // bits 0..coalesce_bits-1 are the contiguous low bits); qb[b] is its
        // qubit.  Shared-memory positions pos[q] start in the same order.
        PassDesc pd{};
        std::vector<int> qb, pos(n, -1);
        int k = 0;
        for (int pb = 0; pb < n; ++pb) {
            const int q = who[pb];
            if ((L >> q) & 1u) {
                pos[q] = (int)qb.size();
                pd.gl[qb.size()] = 1u << pb;
                qb.push_back(q);
            } else {
                pd.gt[k++] = 1u << pb;
            }
        }
        pd.t = t;
        pd.n_tile_bits = n - t;
        pd.local_mask = L;
        // Stages the first `keep` taken ops at positions `ps` (a pass holds at
        // most kPassStages stages and kPassOps group ops); a leading stage
        // without ops is only a permutation and is folded into the tile load
        // (and the reverse pass's tile store).  Returns whether it fits.
        const size_t st0 = P->stages.size(), op0 = P->ops.size();
        auto stage_with = [&](const std::vector<int> &ps, size_t keep) {
            P->stages.resize(st0);
            P->perm_cols.resize(st0);
            P->ops.resize(op0);
            pd.stage_begin = (int)st0;
            std::vector<LOp> sub;
            for (size_t i = 0; i < keep; ++i) sub.push_back(F.lops[taken[i]]);
            stage_lops(sub, ps, t, reg_bits, swz_bits, P, true);
            pd.stage_end = (int)P->stages.size();
            for (int bb = 0; bb < t; ++bb) pd.ldperm[bb] = swizzle(1u << ps[qb[bb]], swz_bits);
            const Stage &s0 = P->stages[pd.stage_begin];
            if (s0.op_begin == s0.op_end && pd.stage_end - pd.stage_begin > 1) {
                const std::vector<uint32_t> &col = P->perm_cols[pd.stage_begin];
                for (int bb = 0; bb < t; ++bb) pd.ldperm[bb] = swizzle(col[ps[qb[bb]]], swz_bits);
                P->stages.erase(P->stages.begin() + pd.stage_begin);
                P->perm_cols.erase(P->perm_cols.begin() + pd.stage_begin);
                --pd.stage_end;
            }
            int nu = 0;
            for (int si = pd.stage_begin; si < pd.stage_end; ++si) nu += P->stages[si].n_u1;
            pd.n_u1 = nu;
            return pd.stage_end - pd.stage_begin <= kPassStages && nu <= kPassOps;
        };
        // An over-long pass keeps a prefix of the taken ops (a prefix in
        // circuit order is closed under dependencies); the rest go back to
        // the pending list.
        size_t keep = taken.size();
        while (!stage_with(pos, keep) && keep > 1) keep = keep * 3 / 4;
        if (pd.stage_end - pd.stage_begin > kPassStages || pd.n_u1 > kPassOps)
            return "internal: a tile pass exceeds the stage or op limit";
        for (size_t i = keep; i < taken.size(); ++i) rest.push_back(taken[i]);
        std::sort(rest.begin(), rest.end());
        // Relabel on the way out: the local qubits that the remaining ops
        // need first take the low bits; the qubits they displace take the
        // bits these leave (all within the tile, so the stored tile covers
        // the same addresses).
        std::vector<int> nwho = who;
        if (relabel && !rest.empty()) {
            std::vector<int> want;
            for (size_t i = 0; i < rest.size() && (int)want.size() < coalesce_bits; ++i) {
                const LOp &o = F.lops[rest[i]];
                const int qs[2] = {o.a, o.kind == 0 ? -1 : o.b};
                for (int q : qs)
                    if (q >= 0 && ((L >> q) & 1u) && (int)want.size() < coalesce_bits &&
                        std::find(want.begin(), want.end(), q) == want.end())
                        want.push_back(q);
            }
            for (int q : want) {
                if (phys[q] < coalesce_bits) continue;
                int lb = -1;  // a low bit whose qubit is not wanted there
                for (int x = 0; x < coalesce_bits && lb < 0; ++x)
                    if (std::find(want.begin(), want.end(), nwho[x]) == want.end()) lb = x;
                if (lb < 0) break;
                const int hb = phys[q], out = nwho[lb];
                nwho[lb] = q;
                nwho[hb] = out;
            }
            // Shared-memory positions whose residues mod swz_bits differ
            // across the qubits of the low bits before the pass (the lanes
            // of the tile load) and across those after it (the lanes of the
            // tile store), so both hit distinct banks; re-staged with them
            // when the pass still fits.
            if (swz_bits == coalesce_bits) {
                const int w = swz_bits;
                std::vector<int> res(n, -1), lowin, lowout;
                for (int x = 0; x < w; ++x) {
                    lowin.push_back(who[x]);
                    lowout.push_back(nwho[x]);
                }
                std::vector<bool> used_in(w, false), used_out(w, false);
                for (int q : lowin)
                    if (std::find(lowout.begin(), lowout.end(), q) != lowout.end())
                        for (int r = 0; r < w; ++r)
                            if (!used_in[r] && !used_out[r]) {
                                res[q] = r;
                                used_in[r] = used_out[r] = true;
                                break;
                            }
                for (int q : lowin)
                    if (res[q] < 0)
                        for (int r = 0; r < w; ++r)
                            if (!used_in[r]) {
                                res[q] = r;
                                used_in[r] = true;
                                break;
                            }
                for (int q : lowout)
                    if (res[q] < 0)
                        for (int r = 0; r < w; ++r)
                            if (!used_out[r]) {
                                res[q] = r;
                                used_out[r] = true;
                                break;
                            }
                std::vector<int> pos2(n, -1);
                std::vector<bool> taken_pos(t, false);
                bool ok = true;
                for (int q : qb)
                    if (res[q] >= 0) {
                        int pp = -1;
                        for (int c2 = res[q]; c2 < t && pp < 0; c2 += w)
                            if (!taken_pos[c2]) pp = c2;
                        if (pp < 0) ok = false;
                        else {
                            pos2[q] = pp;
                            taken_pos[pp] = true;
                        }
                    }
                for (int q : qb)
                    if (pos2[q] < 0)
                        for (int pp = 0; pp < t; ++pp)
                            if (!taken_pos[pp]) {
                                pos2[q] = pp;
                                taken_pos[pp] = true;
                                break;
                            }
                if (ok && pos2 != pos) {
                    if (stage_with(pos2, keep)) pos = pos2;
                    else stage_with(pos, keep);
                }
            }
            for (int q = 0; q < n; ++q) phys[nwho[q]] = q;
        }
        // The store writes to tile bit bb the shared-memory position of the
        // qubit that now lives in its index bit.
        std::vector<uint32_t> stp(t);
        for (int bb = 0; bb < t; ++bb)
            stp[bb] = swizzle(1u << pos[nwho[__builtin_ctz(pd.gl[bb])]], swz_bits);
        who.swap(nwho);
        P->stperm.push_back(stp);
        P->passes.push_back(pd);
        pending.swap(rest);
    }
    P->layout = phys;
    return "";
}

// Kernel descriptors of every pass of a tile plan (amplitudes of csz bytes).
std::string build_tile_passes(const HostProgram &P, int csz, std::vector<TilePass> *out) {
    out->clear();
    const int R = P.R, w = P.swz_bits;
    for (const PassDesc &pd : P.passes) {
        TilePass tp{};
        tp.t = pd.t;
        tp.R = R;
        tp.n_stages = pd.stage_end - pd.stage_begin;
        tp.n_tile_bits = pd.n_tile_bits;
        if (tp.n_stages > kPassStages) return "too many stages in a tile pass";
        if (pd.t - R < 5) return "tile passes need at least 32 threads (tile_bits - reg_bits >= 5)";
        for (int b = 0; b < pd.t; ++b) {
            tp.gl[b] = pd.gl[b];
            tp.ldperm[b] = pd.ldperm[b] * (uint32_t)csz;
            tp.nat[b] = (P.stperm.empty() ? swizzle(1u << b, w) : P.stperm[&pd - P.passes.data()][b]) *
                        (uint32_t)csz;
        }
        uint32_t acc = 0;
        for (int k = 0; k < pd.n_tile_bits; ++k) {
            acc ^= pd.gt[k];
            tp.gpre[k] = acc;
        }
        int u = 0;
        for (int si = 0; si < tp.n_stages; ++si) {
            const Stage &sg = P.stages[pd.stage_begin + si];
            TileStage &ts = tp.st[si];
            for (int i = 0; i < kRMax; ++i) {
                ts.op[i] = -1;
                ts.ldq[i] = i < R ? sg.ldq[i] * (uint32_t)csz : 0u;
                ts.stq[i] = i < R ? sg.stq[i] * (uint32_t)csz : 0u;
            }
            for (int k = 0; k < pd.t - R; ++k) {
                ts.ldt[k] = sg.ldt[k] * (uint32_t)csz;
                ts.stt[k] = sg.stt[k] * (uint32_t)csz;
            }
            for (int oi = sg.op_begin; oi < sg.op_end; ++oi) {
                const Op &op = P.ops[oi];
                if (op.kind != OP_U1) return "tile pass stage holds a non-group op";
                if (op.a < 0 || op.a >= R || ts.op[op.a] >= 0)
                    return "tile pass stage holds two ops on one register bit";
                if (u >= kPassOps) return "too many ops in a tile pass";
                ts.op[op.a] = u;
                tp.grp[u] = op.group;
                const Group &gr = P.groups[op.group];
                if (gr.real) tp.real_mask |= 1ull << u;
                if (gr.has_param) {
                    tp.param_mask |= 1ull << u;
                    int n_par = 0, last_par = -1;
                    for (int m = gr.m_begin; m < gr.m_end; ++m) {
                        const Member &mb = P.members[m];
                        if (mb.kind <= M_RZ && mb.param >= 0) {
                            ++n_par;
                            last_par = m;
                        }
                    }
                    if (n_par == 1 && last_par == gr.m_end - 1) {
                        const int k = P.members[last_par].kind;
                        tp.fmode[u] = (int8_t)(k == M_RY ? 1 : (k == M_RX ? 2 : 3));
                    }
                }
                ++u;
            }
        }
        tp.n_ops = u;
        tp.all_single = 1;
        for (int v = 0; v < u; ++v)
            if (((tp.param_mask >> v) & 1ull) && tp.fmode[v] == 0) tp.all_single = 0;
        out->push_back(tp);
    }
    return "";
}

std::string plan_h_passes(const HostObservable &h, int tile_bits, int coalesce_bits,
                          HostHPlan *out) {
    const int n = h.n, t = tile_bits;
    if (t < coalesce_bits + 1 || t > n || t > kTileBitsMax) return "bad tile_bits for H passes";
    *out = HostHPlan();
    const uint32_t forced = (1u << coalesce_bits) - 1u;
    std::vector<int> pending(h.tgroups.size());
    for (size_t i = 0; i < pending.size(); ++i) pending[i] = (int)i;
    while (!pending.empty()) {
        uint32_t L = forced;
        std::vector<int> taken, rest;
        std::vector<int> far;  // flip masks that fit no tile: partners from global memory
        for (int gi : pending) {
            const uint32_t x = h.tgroups[gi].x;
            if (__builtin_popcount(forced | x) > t) {
                far.push_back(gi);
            } else if (__builtin_popcount(L | x) <= t) {
                L |= x;
                taken.push_back(gi);
            } else {
                rest.push_back(gi);
            }
        }
        if (taken.empty() && far.empty()) return "internal: H pass planner made no progress";
        for (int gi : far) taken.push_back(gi);
        for (int q = 0; __builtin_popcount(L) < t && q < n; ++q) L |= 1u << q;
        HPass P{};
        P.t = t;
        P.n_tile_bits = n - t;
        P.first = out->passes.empty() ? 1 : 0;
        P.R = h_reg_bits(t);
        std::vector<int> pos(n, -1);
        int b = 0, k = 0;
        uint32_t acc = 0;
        for (int q = 0; q < n; ++q) {
            if ((L >> q) & 1u) {
                pos[q] = b;
                P.gl[b++] = 1u << q;
            } else {
                acc ^= 1u << q;
                P.gpre[k++] = acc;
            }
        }
        auto local = [&](uint32_t m) {
            uint32_t r = 0;
            for (int q = 0; q < n; ++q)
                if (((m >> q) & 1u) && pos[q] >= 0) r |= 1u << pos[q];
            return r;
        };
        out->g_begin.push_back((int)out->groups.size());
        out->c_begin.push_back((int)out->classes.size());
        out->t_begin.push_back((int)out->terms.size());
        out->r_begin.push_back((int)out->rows.size());
        const int g0 = (int)out->groups.size(), c0 = (int)out->classes.size(),
                  t0 = (int)out->terms.size(), r0 = (int)out->rows.size();
        const uint32_t tmask = (1u << (t - P.R)) - 1u;
        for (int gi : taken) {
            const TermGroup &tg = h.tgroups[gi];
            HGroup G{};
            G.xl = local(tg.x);
            const uint32_t xnl = tg.x & ~L;
            G.xfar = xnl ? tg.x : 0u;
            G.c_begin = (int)out->classes.size() - c0;
            std::vector<int> order;
            for (int ti = tg.t_begin; ti < tg.t_end; ++ti) order.push_back(ti);
            // by the Z mask's thread bits, then its register bits
            std::stable_sort(order.begin(), order.end(), [&](int a, int bb) {
                const uint32_t za = local(h.terms[a].z), zb = local(h.terms[bb].z);
                if ((za & tmask) != (zb & tmask)) return (za & tmask) < (zb & tmask);
                return za < zb;
            });
            for (size_t i = 0; i < order.size(); ++i) {
                const Term &tm = h.terms[order[i]];
                const uint32_t zl = local(tm.z);
                if (i == 0 || zl != out->classes.back().zl ||
                    (int)out->classes.size() - c0 == G.c_begin) {
                    HClass C{};
                    C.zl = zl;
                    C.xnl = xnl;
                    C.xl = G.xl;
                    C.t_begin = (int)out->terms.size() - t0;
                    out->classes.push_back(C);
                }
                HTerm ht{};
                ht.z = tm.z;
                ht.phase = tm.phase;
                ht.coeff = tm.coeff;
                out->terms.push_back(ht);
                out->classes.back().t_end = (int)out->terms.size() - t0;
            }
            G.c_end = (int)out->classes.size() - c0;
            for (int c = G.c_begin; c < G.c_end; ++c)
                G.kact |= out->classes[(size_t)(c0 + c)].zl >> (t - P.R);
            // rows: the runs of classes with the same Z mask on the thread bits
            G.r_begin = G.r_end = (int)out->rows.size() - r0;
            if (G.kact)
                for (int c = G.c_begin; c < G.c_end; ++c) {
                    const uint32_t zt = out->classes[(size_t)(c0 + c)].zl & tmask;
                    if (c == G.c_begin || zt != out->rows.back().zt) {
                        HRow rw{};
                        rw.zt = zt;
                        rw.c_begin = c;
                        out->rows.push_back(rw);
                    }
                    out->rows.back().c_end = c + 1;
                }
            G.r_end = (int)out->rows.size() - r0;
            out->groups.push_back(G);
        }
        P.real = 1;
        for (size_t i = (size_t)t0; i < out->terms.size(); ++i) P.real &= (out->terms[i].phase & 1) == 0;
        P.n_groups = (int)out->groups.size() - g0;
        P.n_classes = (int)out->classes.size() - c0;
        P.n_terms = (int)out->terms.size() - t0;
        P.n_rows = (int)out->rows.size() - r0;
        out->passes.push_back(P);
        pending.swap(rest);
    }
    out->g_begin.push_back((int)out->groups.size());
    out->c_begin.push_back((int)out->classes.size());
    out->t_begin.push_back((int)out->terms.size());
    out->r_begin.push_back((int)out->rows.size());
    return "";
}

std::string plan_observable(const sv_pauli_sum &h, int n, int swz_bits, HostObservable *out) {
    if (h.n_terms < 0) return "negative n_terms";
    if (h.n_terms > 0 && (!h.x_mask || !h.z_mask || !h.coeff)) return "observable arrays missing";
    if (h.n_qubits != n) return "observable qubit count differs from the state's";
    const uint64_t lim = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    *out = HostObservable();
    out->n = n;
    std::vector<uint32_t> xs;
    std::vector<std::vector<Term>> per;
    std::unordered_map<uint32_t, int> idx;
    for (int t = 0; t < h.n_terms; ++t) {
        if ((h.x_mask[t] & ~lim) || (h.z_mask[t] & ~lim))
            return "term " + std::to_string(t) + ": mask has bits beyond n_qubits";
        const uint32_t x = (uint32_t)h.x_mask[t], z = (uint32_t)h.z_mask[t];
        auto it = idx.find(x);
        int gi;
        if (it == idx.end()) {
            gi = (int)xs.size();
            idx[x] = gi;
            xs.push_back(x);
            per.emplace_back();
        } else {
            gi = it->second;
        }
        Term tm{};
        tm.z = z;
        tm.phase = __builtin_popcount(x & z) & 3;
        tm.coeff = h.coeff[t];
        per[gi].push_back(tm);
    }
    for (size_t g = 0; g < xs.size(); ++g) {
        TermGroup tg{};
        tg.x = xs[g];
        tg.sx = swizzle(xs[g], swz_bits);
        tg.t_begin = (int)out->terms.size();
        for (const Term &tm : per[g]) out->terms.push_back(tm);
        tg.t_end = (int)out->terms.size();
        out->tgroups.push_back(tg);
    }
    return "";
}

uint64_t hash_circuit(const sv_circuit &c) {
    uint64_t h = 0x12345678abcdefull;
    h = mix(h, (uint64_t)c.n_qubits);
    h = mix(h, (uint64_t)c.n_gates);
    h = mix(h, (uint64_t)c.n_params);
    h = mix(h, (uint64_t)c.input_dim);
    for (int g = 0; g < c.n_gates; ++g) {
        const sv_gate &G = c.gates[g];
        uint64_t a;
        std::memcpy(&a, &G.angle, sizeof a);
        h = mix(h, (uint64_t)(uint32_t)G.op | ((uint64_t)(uint32_t)G.target << 32));
        h = mix(h, (uint64_t)(uint32_t)G.control | ((uint64_t)(uint32_t)G.param << 32));
        h = mix(h, a);
    }
    return h;
}

uint64_t hash_observable(const sv_pauli_sum &o) {
    uint64_t h = 0x2545F4914F6CDD1Dull;
    h = mix(h, (uint64_t)o.n_qubits);
    h = mix(h, (uint64_t)o.n_terms);
    for (int t = 0; t < o.n_terms; ++t) {
        uint64_t a;
        std::memcpy(&a, &o.coeff[t], sizeof a);
        h = mix(h, o.x_mask[t]);
        h = mix(h, o.z_mask[t]);
        h = mix(h, a);
    }
    return h;
}

}  // namespace svk
