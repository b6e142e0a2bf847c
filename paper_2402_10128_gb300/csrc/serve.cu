// Serving loop (placeholder until the batched scheduler lands).
#include "api_internal.h"

using namespace ges;

extern "C" {
ges_status ges_serve_create(ges_ctx*, const ges_params*, int32_t, ges_server** out) {
  if (out) *out = nullptr;
  return fail(GES_ERR_INVALID_ARG, "serving is not available in this build");
}
ges_status ges_serve_add_scene(ges_server*, const ges_scene*, int32_t*) {
  return fail(GES_ERR_INVALID_ARG, "serving is not available in this build");
}
ges_status ges_serve_submit(ges_server*, int32_t, const ges_camera*, float*, uint64_t*) {
  return fail(GES_ERR_INVALID_ARG, "serving is not available in this build");
}
ges_status ges_serve_poll(ges_server*, uint64_t, int64_t, float*) {
  return fail(GES_ERR_INVALID_ARG, "serving is not available in this build");
}
ges_status ges_serve_destroy(ges_server*) { return GES_OK; }
}
