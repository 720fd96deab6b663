#include "dbnet.h"
extern "C" {
int ens_create(const dbnet_graph_t*, const dbnet_region_params_t*, int32_t, const double*,
               const dbnet_options_t*, const dbens_enkf_t*, void*, dbens_t** out) { if (out) *out = nullptr; return DBNET_EUNSUPPORTED; }
int ens_step(dbens_t*, int64_t) { return DBNET_EUNSUPPORTED; }
int ens_assimilate(dbens_t*, const double*, const double*, const double*, double*) { return DBNET_EUNSUPPORTED; }
int ens_read(dbens_t*, double*, double*, double*) { return DBNET_EUNSUPPORTED; }
int ens_member(dbens_t*, int32_t, dbnet_t**) { return DBNET_EUNSUPPORTED; }
void ens_destroy(dbens_t*) {}
}
