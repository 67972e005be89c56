"""B300-native two-stage approximate inverse of discrete FIOs (BF + HSS-ULV).

The compute path is libfio_b300.so (hand-written sm_103a CUDA behind the C ABI
of include/fio.h); this package only marshals arguments.  Importing it fails
if the library has not been built (`python paper_2609_11520_b300/build.py`).
"""
from .api import BF, HSS, Batch, FioError, device_status, entry_error, fio_pcg, fio_solve, set_large_node  # noqa: F401
