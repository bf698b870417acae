// Temporary entry points for calls whose implementation lands in later files.
#include "ec_internal.h"
using namespace ec;
extern "C" {
int ec_batch(ec_ctx *, const ec_field_desc *, int32_t, void *) { set_error("not built yet"); return EC_ERR_UNSUPPORTED; }
int ec_server_create(ec_ctx *, size_t, int32_t, ec_server **) { set_error("not built yet"); return EC_ERR_UNSUPPORTED; }
int ec_server_submit(ec_server *, const ec_field_desc *, uint64_t *) { return EC_ERR_UNSUPPORTED; }
int ec_server_poll(ec_server *, uint64_t, int *, int32_t *) { return EC_ERR_UNSUPPORTED; }
int ec_server_wait(ec_server *, uint64_t, int64_t, int32_t *) { return EC_ERR_UNSUPPORTED; }
int ec_server_stats(ec_server *, double *) { return EC_ERR_UNSUPPORTED; }
int ec_server_destroy(ec_server *) { return EC_ERR_UNSUPPORTED; }
}
