// Ground state on the GPU (fixed-occupation LDA/LSDA SCF).
#include "hp_internal.h"

extern "C" hp_status hp_ground_state(hp_ctx* c, double nelec, int nspin, const int* init_moment, hp_gs_info* info) {
    (void)nelec; (void)nspin; (void)init_moment; (void)info;
    if (!c) return HP_EINVAL;
    c->err = "hp_ground_state: not available yet";
    return HP_ENOTIMPL;
}
