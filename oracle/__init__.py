"""Plain FP64 CPU oracle of the paper's method (arXiv 2511.02700).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the product path.  It
shares no code with the CUDA library; both sides only share the seeded
input generators of ``paper_2511_02700_gb300.workloads``.
"""
from .levy import (NTSModel, char_exponent_1d, levy_density, levy_density_subordinated,
                   model_from_subordinated_bm, put_price_1d, subordinator_from_mean_variance,
                   variance)
from .scheme import (CALL_AVG, PUT_ASSET1, PUT_AVG, Contract, Grid, Precomputed, Scheme,
                     apply_diffusion, cell_average, circulant_product, cell_integral_r2, diffusion_matrix, extend,
                     far_field, greeks, initial_values, jump_direct, jump_fft, midpoints, precompute,
                     r1_moment, sl_interpolate, sl_weights, solve_nonmixed, zones)
from .sensitivities import PARAMS as SENSITIVITY_PARAMS, price_gradient_fd
from .price_space import PriceGrid, PriceScheme, PriceSpaceOperators
