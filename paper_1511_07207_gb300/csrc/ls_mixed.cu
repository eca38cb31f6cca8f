// ls_mixed.cu -- placeholder until the mixed-precision driver lands.
#include "ls_api_internal.h"

namespace lsi {
int mixed_cg_solve(ls_ctx *, int, const double *, int64_t, const double *, double *,
                   const ls_opts *, ls_info *) {
    return LS_ERR_UNSUPPORTED;
}
size_t mixed_workspace_bytes(int, const ls_opts *, bool) { return 0; }
}  // namespace lsi
