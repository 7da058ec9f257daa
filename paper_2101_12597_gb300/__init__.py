"""GB300-native ETDM energy + gradient path (arXiv:2101.12597).

The CUDA library (libetdm.so, C ABI in include/etdm.h) does all the work;
``paper_2101_12597_gb300.etdm`` is its ctypes binding.  Importing this
package loads nothing; ``ETDM(...)`` loads the library and fails loudly if it
is missing.
"""


def __getattr__(name):
    if name in ("ETDM", "EtdmError", "energy_function", "load_library"):
        from . import etdm
        return getattr(etdm, name)
    raise AttributeError(name)
