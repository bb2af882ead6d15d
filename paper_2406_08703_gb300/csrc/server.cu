// Continuous-batching fit server -- placeholder until the scheduler lands.
#include "dlx_common.cuh"
extern "C" {
int dlx_server_create(int, size_t, int, dlx_server **out) { if (out) *out = nullptr; dlx_set_error("server not built"); return DLX_ERR_UNSUPPORTED; }
int dlx_server_destroy(dlx_server *) { return DLX_OK; }
int dlx_submit(dlx_server *, const dlx_request *, uint64_t *) { return DLX_ERR_UNSUPPORTED; }
int dlx_poll(dlx_server *, uint64_t, double, dlx_result *) { return DLX_ERR_UNSUPPORTED; }
int dlx_server_get_stats(dlx_server *, dlx_server_stats *) { return DLX_ERR_UNSUPPORTED; }
int dlx_server_inject_fault(dlx_server *, int) { return DLX_ERR_UNSUPPORTED; }
}
