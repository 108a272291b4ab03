"""GB300 (sm_103a) implementation of the spatiotemporal Hawkes log-likelihood,
its location and parameter gradients, and HMC over event locations
(Holbrook, Ji & Suchard, arXiv 2010.02994).

The computation lives in libhawkes.so (C ABI: include/hawkes.h); this package
only marshals torch tensors into it.
"""
from .api import (HawkesContext, HawkesError, HawkesMwG, hawkes_batch_hmc_trajectory, hawkes_batch_loglik_grad,  # noqa: F401
                  hawkes_loglik,
                  hawkes_bmds_hmc_trajectory, hawkes_bmds_loglik_grad, hawkes_loglik_grad_locations,
                  hawkes_loglik_noalloc,
                  hawkes_self_excitation_prob,
                  hmc_leapfrog_trajectory, params_struct,
                  probe_dfma_rate, probe_exp2_fp64, probe_pipe_rates,
                  version)
from .autograd import HawkesLogLik, hawkes_loglik_autograd  # noqa: F401,E402
