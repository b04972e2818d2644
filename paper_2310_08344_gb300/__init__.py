"""GB300-native Leja exponential-integrator engine (Python binding).

A thin ctypes layer over the C ABI declared in include/lexgb.h: each function
here has the name of the C entry point it calls and only marshals arguments
(torch CUDA tensors or raw device addresses to pointers, numpy arrays to host
pointers).  Every step of the computation runs in the CUDA library
``_lexgb.so``; importing this package without that library raises.
PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

from .binding import (  # noqa: F401
    ADVDIFF,
    ADVDIFF_UP3,
    BURGERS_UP3,
    BURGERS,
    EXPRB32,
    DF64,
    FP64,
    MIXED,
    ROS_EU,
    STATUS,
    Batch,
    Context,
    LexgbError,
    Mlp,
    batch_setup,
    batch_stats,
    batch_step,
    expint_step,
    expint_step_host,
    leja_destroy,
    leja_setup,
    lib,
    lx_controller_classical,
    lx_ctx_autotune,
    lx_ctx_kernel_name,
    lx_ctx_select_kernel,
    lx_ctx_iters_per_launch,
    lx_ctx_set_loop_mode,
    lx_ctx_set_graph_unroll,
    lx_ctx_set_source,
    phi_l_apply_vertical,
    lx_ctx_stats,
    lx_leja_coeff_count,
    lx_leja_coeffs,
    lx_integrate,
    lx_integrate_learned,
    lx_leja_points,
    lx_status_str,
    mlp_forward,
    mlp_forward_host,
    mlp_get_weights,
    mlp_param_count,
    mlp_setup,
    mlp_train_step,
    phi_l_apply,
    phi_l_apply_noalloc,
    power_bound,
    spectral_interval,
)
