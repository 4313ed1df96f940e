"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package draws random numbers and encodes the stored bytes of the data
matrix; it holds no step of the LocalPower method itself (no orthonormalisation
of iterates, no power step, no alignment, no averaging).  Both sides of every
parity check consume the arrays produced here, so they run on the same bytes.
"""
from .spiked import (  # noqa: F401
    partition_sizes,
    spiked_rows,
    gaussian_start,
    haar_columns,
    split_rows,
)
from .lowprec import (  # noqa: F401
    f32_to_bf16_bits,
    f32_to_bf16x2_planes,
    f32_to_e4m3_rowscaled,
    E4M3_MAX,
)
from .configs import CONFIGS, config_schedule, make_config_data  # noqa: F401
