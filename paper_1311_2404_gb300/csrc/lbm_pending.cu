// Entry points whose kernels are not in this build yet: they validate
// nothing and report LBM_EINVAL with a message.
#include <string>

#include "../../include/lbm.h"

static thread_local std::string g_pending_err;

static int pending(const char* what)
{
    g_pending_err = std::string(what) + ": not available in this build";
    return LBM_EINVAL;
}

extern "C" {
int lbm_batch_create(int, const int*, const int*, const double*, int, lbm_batch* out)
{
    if (out) *out = nullptr;
    return pending("lbm_batch_create");
}
int lbm_batch_destroy(lbm_batch) { return LBM_OK; }
const char* lbm_batch_last_error(lbm_batch) { return g_pending_err.c_str(); }
int lbm_batch_set_stream(lbm_batch, void*) { return pending("lbm_batch_set_stream"); }
int lbm_batch_set_geometry(lbm_batch, int, const uint8_t*) { return pending("lbm_batch_set_geometry"); }
int lbm_batch_set_force(lbm_batch, int, double, double) { return pending("lbm_batch_set_force"); }
int lbm_batch_init_equilibrium(lbm_batch, int, const void*, const void*, int)
{
    return pending("lbm_batch_init_equilibrium");
}
int lbm_batch_autotune(lbm_batch) { return pending("lbm_batch_autotune"); }
int lbm_batch_get_config(lbm_batch, int*) { return pending("lbm_batch_get_config"); }
int lbm_batch_step(lbm_batch, int) { return pending("lbm_batch_step"); }
int lbm_batch_get_macro(lbm_batch, int, void*, void*, int) { return pending("lbm_batch_get_macro"); }
int lbm_batch_sync(lbm_batch) { return pending("lbm_batch_sync"); }
long long lbm_batch_launch_count(lbm_batch) { return 0; }
size_t lbm_batch_nodes(lbm_batch) { return 0; }
int lbm_mlp_train(const float*, const double*, int, const double*, float*, float*, void*)
{
    return pending("lbm_mlp_train");
}
int lbm_mlp_grad(const float*, const float*, int, const float*, float*, float*, void*)
{
    return pending("lbm_mlp_grad");
}
int lbm_mlp_forward(const float*, int, const float*, float*, void*) { return pending("lbm_mlp_forward"); }
}
