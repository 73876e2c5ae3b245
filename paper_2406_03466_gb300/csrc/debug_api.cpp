// Test hooks declared in sv_debug.h: host-side planner output, no GPU needed.
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "planner.h"
#include "sv_debug.h"

using namespace svk;

extern "C" {

void sv_debug_sizes(int32_t *sizes) {
    if (!sizes) return;
    sizes[0] = (int32_t)sizeof(Stage);
    sizes[1] = (int32_t)sizeof(Op);
    sizes[2] = (int32_t)sizeof(Group);
    sizes[3] = (int32_t)sizeof(Member);
    sizes[4] = (int32_t)sizeof(TermGroup);
    sizes[5] = (int32_t)sizeof(Term);
    sizes[6] = (int32_t)sizeof(PassDesc);
    sizes[7] = (int32_t)sizeof(TilePass);
}

sv_status sv_debug_plan(const sv_circuit *c, int32_t reg_bits, int32_t fuse, int32_t swz_bits,
                        int32_t *counts, void *stages, void *ops, void *groups, void *members) {
    if (!c || !counts) return SV_ERR_ARG;
    HostProgram h;
    std::string err = plan_circuit(*c, reg_bits, fuse != 0, swz_bits, &h);
    if (!err.empty()) return SV_ERR_ARG;
    counts[0] = (int32_t)h.stages.size();
    counts[1] = (int32_t)h.ops.size();
    counts[2] = (int32_t)h.groups.size();
    counts[3] = (int32_t)h.members.size();
    if (stages) std::memcpy(stages, h.stages.data(), h.stages.size() * sizeof(Stage));
    if (ops) std::memcpy(ops, h.ops.data(), h.ops.size() * sizeof(Op));
    if (groups) std::memcpy(groups, h.groups.data(), h.groups.size() * sizeof(Group));
    if (members) std::memcpy(members, h.members.data(), h.members.size() * sizeof(Member));
    return SV_OK;
}

sv_status sv_debug_passes(const sv_circuit *c, int32_t tile_bits, int32_t coalesce_bits,
                          int32_t reg_bits, int32_t fuse, int32_t swz_bits, int32_t *counts,
                          void *stages, void *ops, void *groups, void *members, void *passes) {
    if (!c || !counts) return SV_ERR_ARG;
    HostProgram h;
    std::string err = plan_passes(*c, tile_bits, coalesce_bits, reg_bits, fuse != 0, swz_bits, &h);
    if (!err.empty()) return SV_ERR_ARG;
    counts[0] = (int32_t)h.stages.size();
    counts[1] = (int32_t)h.ops.size();
    counts[2] = (int32_t)h.groups.size();
    counts[3] = (int32_t)h.members.size();
    counts[4] = (int32_t)h.passes.size();
    if (stages) std::memcpy(stages, h.stages.data(), h.stages.size() * sizeof(Stage));
    if (ops) std::memcpy(ops, h.ops.data(), h.ops.size() * sizeof(Op));
    if (groups) std::memcpy(groups, h.groups.data(), h.groups.size() * sizeof(Group));
    if (members) std::memcpy(members, h.members.data(), h.members.size() * sizeof(Member));
    if (passes) std::memcpy(passes, h.passes.data(), h.passes.size() * sizeof(PassDesc));
    return SV_OK;
}

sv_status sv_debug_tile_passes(const sv_circuit *c, int32_t tile_bits, int32_t reg_bits,
                               int32_t fuse, int32_t dtype, int32_t relabel, int32_t *counts,
                               void *groups, void *members, void *tile_passes, int32_t *layout) {
    if (!c || !counts) return SV_ERR_ARG;
    const bool c128 = dtype == SV_C128;
    HostProgram h;
    std::string err = plan_passes(*c, tile_bits, c128 ? 3 : 4, reg_bits, fuse != 0, c128 ? 3 : 4, &h,
                                  relabel != 0);
    std::vector<TilePass> tp;
    if (err.empty()) err = build_tile_passes(h, c128 ? 16 : 8, &tp);
    if (!err.empty()) return SV_ERR_ARG;
    counts[0] = (int32_t)h.groups.size();
    counts[1] = (int32_t)h.members.size();
    counts[2] = (int32_t)tp.size();
    if (groups) std::memcpy(groups, h.groups.data(), h.groups.size() * sizeof(Group));
    if (members) std::memcpy(members, h.members.data(), h.members.size() * sizeof(Member));
    if (tile_passes) std::memcpy(tile_passes, tp.data(), tp.size() * sizeof(TilePass));
    if (layout)
        for (size_t q = 0; q < h.layout.size(); ++q) layout[q] = h.layout[q];
    return SV_OK;
}

sv_status sv_debug_h_passes(const sv_pauli_sum *h, int32_t tile_bits, int32_t coalesce_bits,
                            int32_t *counts, void *passes, void *groups, void *classes,
                            void *terms, void *rows) {
    if (!h || !counts) return SV_ERR_ARG;
    HostObservable ho;
    std::string err = plan_observable(*h, h->n_qubits, 4, &ho);
    HostHPlan hp;
    if (err.empty()) err = plan_h_passes(ho, tile_bits, coalesce_bits, &hp);
    if (!err.empty()) return SV_ERR_ARG;
    counts[0] = (int32_t)hp.passes.size();
    counts[1] = (int32_t)hp.groups.size();
    counts[2] = (int32_t)hp.classes.size();
    counts[3] = (int32_t)hp.terms.size();
    counts[4] = (int32_t)hp.rows.size();
    if (passes) {
        std::vector<HPass> ps = hp.passes;
        for (size_t i = 0; i < ps.size(); ++i) {  // offsets into the arrays, as pointers
            ps[i].groups = (const HGroup *)(uintptr_t)hp.g_begin[i];
            ps[i].classes = (const HClass *)(uintptr_t)hp.c_begin[i];
            ps[i].terms = (const HTerm *)(uintptr_t)hp.t_begin[i];
            ps[i].rows = (const HRow *)(uintptr_t)hp.r_begin[i];
        }
        std::memcpy(passes, ps.data(), ps.size() * sizeof(HPass));
    }
    if (groups) std::memcpy(groups, hp.groups.data(), hp.groups.size() * sizeof(HGroup));
    if (classes) std::memcpy(classes, hp.classes.data(), hp.classes.size() * sizeof(HClass));
    if (terms) std::memcpy(terms, hp.terms.data(), hp.terms.size() * sizeof(HTerm));
    if (rows) std::memcpy(rows, hp.rows.data(), hp.rows.size() * sizeof(HRow));
    return SV_OK;
}

}  // extern "C"
