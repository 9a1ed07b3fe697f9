"""GB300-native 1D sum-of-exponentials fast Gauss transform.

    u_i = sum_j exp(-(x_i - y_j)^2 / (4 delta)) alpha_j          (eqs. 1.1-1.2)

computed in O(n (M + N)) with the SOE approximation of the Gaussian (eq. 1.3)
and the sorted forward/backward recurrences of Sec. 4.  Every step runs in the
CUDA library libfgt1d.so (C ABI in include/fgt1d.h); this package only marshals
arguments.  Import is lazy: the library is loaded on first use.
"""
from .fgt1d import (Plan, soe_cf, transform, sort_merged, execute_host, wait_host, Workspace, backward,  # noqa: F401
                    GaussTransform, gauss_transform, transform_batched, Geometry,
                    transform_self)
