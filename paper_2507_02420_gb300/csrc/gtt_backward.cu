// Reverse-mode derivative of y = G_N x (no counterpart in the paper).
#include "gtt_plan.h"

using namespace gtt;

extern "C" gtt_status_t gtt_backward(gtt_plan_t P, const void *x_saved, const void *dy, void *dx,
                                     void *dW, gtt_stream_t stream) {
    (void)x_saved; (void)dy; (void)dx; (void)dW; (void)stream;
    if (!P) return set_error(GTT_ERR_INVALID_ARG, "NULL plan");
    return set_error(GTT_ERR_UNSUPPORTED, "gtt_backward is not implemented yet");
}
