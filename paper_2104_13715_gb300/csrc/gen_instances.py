"""Generate the per-kernel-side instantiation units of the fused kernel and the
dispatch table (run after editing VARIANTS; the outputs are committed)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))

# kernel side -> list of tile variants (NW warps, QF output rows per warp in the
# forward pass, PF = 1 to load the next R-row window while the current one is used,
# SPLIT = backward row split: 0 whole rows ceil/floor per warp, 1 equal work
# with the MK % NW last rows split by tile-row slices, 2 own rows (each warp
# every kernel row over its forward rows, g in registers), F2 = 1 for packed float2
# FMAs pairing output rows in the forward; 0 if omitted).
# Variant 0 is the default; the autotuner may pick another at run time.
VARIANTS = {
    1: [(8, 4, 0, 0), (8, 2, 0, 0), (8, 8, 0, 0), (4, 4, 0, 0)],
    3: [(8, 4, 0, 0), (8, 2, 0, 0), (8, 8, 0, 0), (4, 4, 0, 0)],
    5: [(8, 2, 0, 0), (8, 4, 0, 0), (8, 8, 0, 0), (4, 4, 0, 0)],
    7: [(8, 4, 0, 0), (8, 8, 0, 0), (8, 4, 0, 0, 1)],
    9: [(8, 4, 0, 2, 1), (8, 4, 0, 1), (8, 8, 0, 1), (8, 4, 0, 1, 1), (8, 4, 0, 2)],
    11: [(8, 4, 0, 1, 1), (8, 4, 1, 1), (8, 4, 0, 1), (12, 4, 0, 0)],
    13: [(12, 4, 1, 1), (12, 4, 0, 1), (13, 4, 0, 0), (12, 4, 1, 1, 1), (12, 4, 0, 2, 1)],
    15: [(12, 4, 0, 2, 1), (12, 4, 1, 1), (12, 4, 0, 1), (12, 4, 1, 1, 1)],
    17: [(8, 4, 0, 1), (8, 4, 1, 1), (8, 4, 1, 1, 1)],
    19: [(8, 4, 1, 1), (8, 4, 0, 1), (10, 4, 0, 0), (8, 4, 1, 1, 1), (8, 4, 0, 1, 1)],
    21: [(8, 4, 0, 0, 1), (8, 4, 0, 0), (8, 4, 1, 0), (7, 4, 0, 0)],
    23: [(8, 4, 0, 0), (8, 4, 1, 0), (8, 4, 1, 0, 1)],
    25: [(12, 4, 1, 1, 1), (12, 4, 0, 1), (12, 4, 1, 1), (13, 4, 0, 0), (12, 2, 0, 1),
         (12, 4, 0, 1, 1), (13, 4, 0, 0, 1)],
    27: [(8, 4, 0, 2, 1), (9, 4, 0, 0), (9, 4, 1, 0)],
    29: [(8, 4, 0, 2, 1), (10, 4, 0, 0), (10, 4, 1, 0)],
    31: [(8, 4, 0, 0), (8, 4, 1, 0)],
}
GROUPS = [[1, 3, 5, 7], [9, 11], [13, 15], [17], [19], [21], [23], [25], [27], [29], [31]]


def main(out=HERE):
    """Write the instantiation units and dia_dispatch.cu into `out` (by
    default beside this script, replacing the previous units)."""
    for f in os.listdir(out):
        if f.startswith("dia_eval_m") and f.endswith(".cu"):
            os.remove(os.path.join(out, f))
    for grp in GROUPS:
        lines = [f"// Fused evaluation kernels for kernel sides {grp} (generated by gen_instances.py)",
                 '#include "dia_eval_inst.cuh"', ""]
        for mk in grp:
            for v, t in enumerate(VARIANTS[mk]):
                nw, qf, mb, sp = t[:4]
                f2 = t[4] if len(t) > 4 else 0
                lines.append(f"DIA_EVAL_INST({mk}, {v}, {nw}, {qf}, {mb}, {sp}, {f2})")
        with open(os.path.join(out, f"dia_eval_m{grp[0]:02d}.cu"), "w") as fh:
            fh.write("\n".join(lines) + "\n")
    decl, cases = [], []
    for mk, vs in VARIANTS.items():
        for v in range(len(vs)):
            decl.append(f"bool kernel_info_{mk}_{v}(KernelInfo *o);")
        inner = " ".join(f"case {v}: return kernel_info_{mk}_{v}(o);" for v in range(len(vs)))
        cases.append(f"        case {mk}:\n            switch (v) {{ {inner} default: return false; }}")
    counts = ", ".join(f"{{{mk}, {len(vs)}}}" for mk, vs in VARIANTS.items())
    src = f"""// Kernel-side and tile-variant dispatch of the fused evaluation kernels
// (generated by gen_instances.py).
#include <atomic>

#include "dia_dispatch.h"

namespace dia {{

{chr(10).join(decl)}

namespace {{
std::atomic<int> g_selected[kMaxKernelSide + 1];
}}

int kernel_variants(int mk) {{
    switch (mk) {{
{chr(10).join(f"        case {mk}: return {len(vs)};" for mk, vs in VARIANTS.items())}
        default: return 0;
    }}
}}

bool kernel_info_variant(int mk, int v, KernelInfo *o) {{
    switch (mk) {{
{chr(10).join(cases)}
        default: return false;
    }}
}}

bool select_variant(int mk, int v) {{
    if (mk < 1 || mk > kMaxKernelSide || v < 0 || v >= kernel_variants(mk)) return false;
    g_selected[mk].store(v);
    return true;
}}

int selected_variant(int mk) {{
    if (mk < 1 || mk > kMaxKernelSide) return 0;
    return g_selected[mk].load();
}}

bool kernel_info(int mk, KernelInfo *o) {{ return kernel_info_variant(mk, selected_variant(mk), o); }}

}}  // namespace dia
"""
    with open(os.path.join(out, "dia_dispatch.cu"), "w") as fh:
        fh.write(src)


if __name__ == "__main__":
    main()
