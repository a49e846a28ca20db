"""B300-native kernel-style nonholonomic planner (arXiv 2306.01301).

The planner itself is the C-ABI library ``_lib/libnhplan.so`` (CUDA kernels
for sm_103a, declared in ``include/nhplan.h``); ``binding`` is its thin Python
binding and ``scenes`` the seeded synthetic inputs.  Importing the package
loads nothing; the first planner call loads the library and fails loudly if
it is missing or no GPU is present.
"""

MANEUVERS = ("LF", "SF", "RB", "RF", "SB", "LB")  # cycle order, Section XVI.A


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def __getattr__(name):
    if name in ("Planner", "PlanError", "PlanResult", "soft_image", "lib"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
