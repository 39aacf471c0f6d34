"""GB300 (sm_103a) channel-flow DNS environment for wall-blowing drag-reduction control.

The compute path lives in ``libchannel_dns.so`` (CUDA, built by
:func:`paper_2301_09889_gb300.build.build`); :mod:`paper_2301_09889_gb300.native`
is its ctypes binding.
"""

from . import native  # noqa: F401
