// Split-precision Rp->q path on the tcgen05 tensor cores (filled in separately).
#include "scatter.cuh"

size_t tc_state_bytes(const epwi_ctx *c) { return sizeof(double2) * (size_t)c->nRp * c->nm * c->nw; }
void tc_restage(epwi_ctx *, const RestageArgs &) {
    throw EpwiError{EPWI_EUNSUPPORTED, "split-precision path not built"};
}
void tc_scatter(epwi_ctx *, const ScatterArgs &, int64_t) {
    throw EpwiError{EPWI_EUNSUPPORTED, "split-precision path not built"};
}
