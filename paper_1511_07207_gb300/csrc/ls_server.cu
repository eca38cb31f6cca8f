// ls_server.cu -- placeholder until the server lands.
#include "ls_api_internal.h"

extern "C" int ls_server_start(ls_ctx *, const ls_server_cfg *, ls_server **) { return LS_ERR_UNSUPPORTED; }
extern "C" int ls_server_submit(ls_server *, const ls_system *, uint64_t *) { return LS_ERR_UNSUPPORTED; }
extern "C" int ls_server_poll(ls_server *, uint64_t, int *, ls_info *) { return LS_ERR_UNSUPPORTED; }
extern "C" int ls_server_stop(ls_server *) { return LS_ERR_UNSUPPORTED; }
