"""GB300-native exact triangle counting: filtered, degree-oriented set
intersection (Wang, Wang, Yang, Owens, HPGP'16, Sec. 3.2 and Alg. 2).

Subpackages:
  * ``binding``  -- ctypes binding of ``libtc.so`` (the C ABI of include/tc.h)
  * ``gen``      -- seeded synthetic graph generators (input data only)

``binding`` is imported on demand so that the generators can be used on
machines without the CUDA library.
"""
__all__ = ["binding", "gen"]
