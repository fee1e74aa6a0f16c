// Pollution-game solver (placeholder until the device iteration lands).
#include "cheb_internal.cuh"

using namespace cheb;

extern "C" cheb_status game_solve(cheb_ctx *ctx, int32_t batch, const cheb_game_params *params,
                                  const cheb_game_opts *opts, cheb_game_result *res, void *stream)
{
    (void)ctx; (void)batch; (void)params; (void)opts; (void)res; (void)stream;
    return fail(CHEB_EUNSUPPORTED, "game_solve: not built yet");
}
