// placeholder, replaced by the tcgen05 engine
#include "common.h"
namespace dcsd {
dcsd_status tc_init(Ctx* c) { (void)c; return DCSD_OK; }
void tc_free(Ctx* c) { (void)c; }
dcsd_status einsum_tc(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B, double beta,
                      const TV& C, int nsplit) {
    (void)nsplit;
    return einsum64(c, spec, alpha, A, B, beta, C);
}
}  // namespace dcsd
