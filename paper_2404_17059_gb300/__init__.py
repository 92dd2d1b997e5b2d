"""GB300-native Monte Carlo engine for the IC and LT diffusion models.

``binding`` exposes the C ABI of libcnd (include/cnd.h) under the same names;
``inputs`` builds seeded synthetic workloads.
"""
from .binding import (  # noqa: F401
    CndError, CndGraph, SimResult, cnd_graph_create, cnd_graph_destroy, cnd_graph_info, cnd_ic_simulate,
    cnd_lt_simulate, cnd_ic_simulate_ex, cnd_lt_simulate_ex, cnd_lt_weights_wc, cnd_philox4x32_10,
    cnd_last_error, cnd_sim_opts_init, cnd_ic_simulate_noalloc, cnd_ic_simulate_batch, cnd_lt_simulate_batch, cnd_autotune, cnd_ic_im_celf, cnd_lt_im_celf, ImResult, CndSur, cnd_sur_create, cnd_sur_destroy,
    cnd_sur_set_params, cnd_sur_get_params, cnd_sur_forward, cnd_sur_loss_grad, cnd_sur_adam, cnd_sur_scores, cnd_sur_onehop,
    cnd_sur_train, cnd_ic_im_screened, cnd_philox_rate, cnd_random_access_rate, CND_SUR_N_PARAMS, CND_STATS_COUNT, CND_STATS_TIMING, CND_OK, CND_EINVAL, CND_ENOMEM, CND_ECUDA, CND_ELIMIT, CND_ETIMEOUT,
    CND_EOVERFLOW,
)
