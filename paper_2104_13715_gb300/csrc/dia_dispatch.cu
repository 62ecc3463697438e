// Kernel-side dispatch for the fused evaluation kernels.
#include "dia_dispatch.h"

namespace dia {

#define DIA_DECL(MKV) bool kernel_info_##MKV(KernelInfo *o);
DIA_DECL(1) DIA_DECL(3) DIA_DECL(5) DIA_DECL(7) DIA_DECL(9) DIA_DECL(11) DIA_DECL(13)
DIA_DECL(15) DIA_DECL(17) DIA_DECL(19) DIA_DECL(21) DIA_DECL(23) DIA_DECL(25) DIA_DECL(27)
DIA_DECL(29) DIA_DECL(31)
#undef DIA_DECL

bool kernel_info(int mk, KernelInfo *o) {
    switch (mk) {
#define DIA_CASE(MKV) \
    case MKV: return kernel_info_##MKV(o);
        DIA_CASE(1) DIA_CASE(3) DIA_CASE(5) DIA_CASE(7) DIA_CASE(9) DIA_CASE(11) DIA_CASE(13)
        DIA_CASE(15) DIA_CASE(17) DIA_CASE(19) DIA_CASE(21) DIA_CASE(23) DIA_CASE(25)
        DIA_CASE(27) DIA_CASE(29) DIA_CASE(31)
#undef DIA_CASE
        default: return false;
    }
}

}  // namespace dia
