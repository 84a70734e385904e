"""GB300-native element integration for higher-order prismatic finite elements.

The hot path of Kruzel & Banas (numerical integration of element stiffness
matrices and load vectors, Sec. 2, Algorithm 1) as hand-written CUDA for
sm_103a behind the C ABI in include/fei.h.  ``inputs`` (seeded synthetic
workloads) needs neither torch nor the library; the kernel entry points
(``fei_integrate``, ``fei_integrate_backward``, ``fei_reference_create``,
``fei_plan_offsets``, ``integrate``) load the compiled library on first use
and raise ImportError if it is not built.
"""
from . import inputs  # noqa: F401

_API_NAMES = ("fei_integrate", "fei_integrate_backward", "fei_reference_create",
              "fei_plan_offsets", "integrate", "Reference", "Layout", "uniform_layout", "nsh", "nq", "Plan",
              "fei_integrate_backward_quadratic", "fei_status_summary", "Assembly", "Pipeline")


def __getattr__(name):
    if name in _API_NAMES:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
