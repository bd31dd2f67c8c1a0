"""FP64 CPU oracle for the GSW-MTP loop -- test infrastructure only.

Imported by the tests, the package smoke check and the benchmark's CPU
baseline leg; never by the library's product path.
"""
from .gsw_mtp import *  # noqa: F401,F403
