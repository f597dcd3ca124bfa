"""GB300-native FFT-based Yamamoto estimator of the power-spectrum multipoles
P_0, P_2, P_4 with a varying line of sight (Bianchi et al. 2015).

The work runs in libystat.so (CUDA, sm_103a) behind the C ABI of include/ystat.h;
``ystat.Plan`` is its thin Python binding.
"""
from .ystat import MLP_PARAMS, Batch, Mlp, Plan, Result, YstatError, header_functions, load_library, make_config, parse_row, sum_gal, wedges

__all__ = ["MLP_PARAMS", "Batch", "Mlp", "Plan", "Result", "YstatError", "header_functions", "load_library", "make_config", "parse_row", "sum_gal", "wedges"]
