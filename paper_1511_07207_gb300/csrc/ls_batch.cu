// ls_batch.cu -- placeholder until the batched driver and the server land.
#include "ls_api_internal.h"

namespace lsi {
void extra_destroy(ls_ctx *) {}
}  // namespace lsi

extern "C" int ls_batch_solve(ls_ctx *, int, const ls_system *, ls_info *) { return LS_ERR_UNSUPPORTED; }
extern "C" int ls_server_start(ls_ctx *, const ls_server_cfg *, ls_server **) { return LS_ERR_UNSUPPORTED; }
extern "C" int ls_server_submit(ls_server *, const ls_system *, uint64_t *) { return LS_ERR_UNSUPPORTED; }
extern "C" int ls_server_poll(ls_server *, uint64_t, int *, ls_info *) { return LS_ERR_UNSUPPORTED; }
extern "C" int ls_server_stop(ls_server *) { return LS_ERR_UNSUPPORTED; }
