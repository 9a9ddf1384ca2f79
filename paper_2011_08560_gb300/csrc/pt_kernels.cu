// pt_kernels.cu -- parallel tempering (second kernel); filled in below.
#include <cuda_runtime.h>

#include "eamc.h"
#include "eamc_ctx.cuh"

struct PtState {};

void pt_release(ea_ctx *ctx) {
    if (!ctx || !ctx->pt) return;
    delete ctx->pt;
    ctx->pt = nullptr;
}
