"""GB300-native semi-discrete optimal transport (Laguerre cells + damped Newton).

The compute path is libsdot.so (hand-written CUDA for sm_103a behind the C ABI of
include/sdot.h); ``binding`` marshals arguments to it. ``ics`` builds the seeded
synthetic inputs. Importing the package loads nothing; ``binding`` loads the
library on first use and raises if it is missing.
"""
__all__ = ["binding", "ics", "build"]
