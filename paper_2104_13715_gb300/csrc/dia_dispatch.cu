// Kernel-side and tile-variant dispatch of the fused evaluation kernels
// (generated by gen_instances.py).
#include <atomic>

#include "dia_dispatch.h"

namespace dia {

bool kernel_info_1_0(KernelInfo *o);
bool kernel_info_1_1(KernelInfo *o);
bool kernel_info_1_2(KernelInfo *o);
bool kernel_info_1_3(KernelInfo *o);
bool kernel_info_3_0(KernelInfo *o);
bool kernel_info_3_1(KernelInfo *o);
bool kernel_info_3_2(KernelInfo *o);
bool kernel_info_3_3(KernelInfo *o);
bool kernel_info_5_0(KernelInfo *o);
bool kernel_info_5_1(KernelInfo *o);
bool kernel_info_5_2(KernelInfo *o);
bool kernel_info_5_3(KernelInfo *o);
bool kernel_info_7_0(KernelInfo *o);
bool kernel_info_7_1(KernelInfo *o);
bool kernel_info_7_2(KernelInfo *o);
bool kernel_info_9_0(KernelInfo *o);
bool kernel_info_9_1(KernelInfo *o);
bool kernel_info_9_2(KernelInfo *o);
bool kernel_info_9_3(KernelInfo *o);
bool kernel_info_9_4(KernelInfo *o);
bool kernel_info_11_0(KernelInfo *o);
bool kernel_info_11_1(KernelInfo *o);
bool kernel_info_11_2(KernelInfo *o);
bool kernel_info_11_3(KernelInfo *o);
bool kernel_info_13_0(KernelInfo *o);
bool kernel_info_13_1(KernelInfo *o);
bool kernel_info_13_2(KernelInfo *o);
bool kernel_info_13_3(KernelInfo *o);
bool kernel_info_13_4(KernelInfo *o);
bool kernel_info_15_0(KernelInfo *o);
bool kernel_info_15_1(KernelInfo *o);
bool kernel_info_15_2(KernelInfo *o);
bool kernel_info_15_3(KernelInfo *o);
bool kernel_info_17_0(KernelInfo *o);
bool kernel_info_17_1(KernelInfo *o);
bool kernel_info_17_2(KernelInfo *o);
bool kernel_info_19_0(KernelInfo *o);
bool kernel_info_19_1(KernelInfo *o);
bool kernel_info_19_2(KernelInfo *o);
bool kernel_info_19_3(KernelInfo *o);
bool kernel_info_19_4(KernelInfo *o);
bool kernel_info_21_0(KernelInfo *o);
bool kernel_info_21_1(KernelInfo *o);
bool kernel_info_21_2(KernelInfo *o);
bool kernel_info_21_3(KernelInfo *o);
bool kernel_info_23_0(KernelInfo *o);
bool kernel_info_23_1(KernelInfo *o);
bool kernel_info_23_2(KernelInfo *o);
bool kernel_info_25_0(KernelInfo *o);
bool kernel_info_25_1(KernelInfo *o);
bool kernel_info_25_2(KernelInfo *o);
bool kernel_info_25_3(KernelInfo *o);
bool kernel_info_25_4(KernelInfo *o);
bool kernel_info_25_5(KernelInfo *o);
bool kernel_info_25_6(KernelInfo *o);
bool kernel_info_27_0(KernelInfo *o);
bool kernel_info_27_1(KernelInfo *o);
bool kernel_info_27_2(KernelInfo *o);
bool kernel_info_29_0(KernelInfo *o);
bool kernel_info_29_1(KernelInfo *o);
bool kernel_info_29_2(KernelInfo *o);
bool kernel_info_31_0(KernelInfo *o);
bool kernel_info_31_1(KernelInfo *o);

namespace {
std::atomic<int> g_selected[kMaxKernelSide + 1];
}

int kernel_variants(int mk) {
    switch (mk) {
        case 1: return 4;
        case 3: return 4;
        case 5: return 4;
        case 7: return 3;
        case 9: return 5;
        case 11: return 4;
        case 13: return 5;
        case 15: return 4;
        case 17: return 3;
        case 19: return 5;
        case 21: return 4;
        case 23: return 3;
        case 25: return 7;
        case 27: return 3;
        case 29: return 3;
        case 31: return 2;
        default: return 0;
    }
}

bool kernel_info_variant(int mk, int v, KernelInfo *o) {
    switch (mk) {
        case 1:
            switch (v) { case 0: return kernel_info_1_0(o); case 1: return kernel_info_1_1(o); case 2: return kernel_info_1_2(o); case 3: return kernel_info_1_3(o); default: return false; }
        case 3:
            switch (v) { case 0: return kernel_info_3_0(o); case 1: return kernel_info_3_1(o); case 2: return kernel_info_3_2(o); case 3: return kernel_info_3_3(o); default: return false; }
        case 5:
            switch (v) { case 0: return kernel_info_5_0(o); case 1: return kernel_info_5_1(o); case 2: return kernel_info_5_2(o); case 3: return kernel_info_5_3(o); default: return false; }
        case 7:
            switch (v) { case 0: return kernel_info_7_0(o); case 1: return kernel_info_7_1(o); case 2: return kernel_info_7_2(o); default: return false; }
        case 9:
            switch (v) { case 0: return kernel_info_9_0(o); case 1: return kernel_info_9_1(o); case 2: return kernel_info_9_2(o); case 3: return kernel_info_9_3(o); case 4: return kernel_info_9_4(o); default: return false; }
        case 11:
            switch (v) { case 0: return kernel_info_11_0(o); case 1: return kernel_info_11_1(o); case 2: return kernel_info_11_2(o); case 3: return kernel_info_11_3(o); default: return false; }
        case 13:
            switch (v) { case 0: return kernel_info_13_0(o); case 1: return kernel_info_13_1(o); case 2: return kernel_info_13_2(o); case 3: return kernel_info_13_3(o); case 4: return kernel_info_13_4(o); default: return false; }
        case 15:
            switch (v) { case 0: return kernel_info_15_0(o); case 1: return kernel_info_15_1(o); case 2: return kernel_info_15_2(o); case 3: return kernel_info_15_3(o); default: return false; }
        case 17:
            switch (v) { case 0: return kernel_info_17_0(o); case 1: return kernel_info_17_1(o); case 2: return kernel_info_17_2(o); default: return false; }
        case 19:
            switch (v) { case 0: return kernel_info_19_0(o); case 1: return kernel_info_19_1(o); case 2: return kernel_info_19_2(o); case 3: return kernel_info_19_3(o); case 4: return kernel_info_19_4(o); default: return false; }
        case 21:
            switch (v) { case 0: return kernel_info_21_0(o); case 1: return kernel_info_21_1(o); case 2: return kernel_info_21_2(o); case 3: return kernel_info_21_3(o); default: return false; }
        case 23:
            switch (v) { case 0: return kernel_info_23_0(o); case 1: return kernel_info_23_1(o); case 2: return kernel_info_23_2(o); default: return false; }
        case 25:
            switch (v) { case 0: return kernel_info_25_0(o); case 1: return kernel_info_25_1(o); case 2: return kernel_info_25_2(o); case 3: return kernel_info_25_3(o); case 4: return kernel_info_25_4(o); case 5: return kernel_info_25_5(o); case 6: return kernel_info_25_6(o); default: return false; }
        case 27:
            switch (v) { case 0: return kernel_info_27_0(o); case 1: return kernel_info_27_1(o); case 2: return kernel_info_27_2(o); default: return false; }
        case 29:
            switch (v) { case 0: return kernel_info_29_0(o); case 1: return kernel_info_29_1(o); case 2: return kernel_info_29_2(o); default: return false; }
        case 31:
            switch (v) { case 0: return kernel_info_31_0(o); case 1: return kernel_info_31_1(o); default: return false; }
        default: return false;
    }
}

bool select_variant(int mk, int v) {
    if (mk < 1 || mk > kMaxKernelSide || v < 0 || v >= kernel_variants(mk)) return false;
    g_selected[mk].store(v);
    return true;
}

int selected_variant(int mk) {
    if (mk < 1 || mk > kMaxKernelSide) return 0;
    return g_selected[mk].load();
}

bool kernel_info(int mk, KernelInfo *o) { return kernel_info_variant(mk, selected_variant(mk), o); }

}  // namespace dia
