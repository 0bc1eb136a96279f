"""GB300-native (sm_103a) hot path of relativistic Fock-space coupled cluster.

``expgb`` is the ctypes binding of the C ABI in include/exp.h (libexpgb.so, built
by ``build.build()``); ``synthetic`` holds the seeded input draws.  Importing the
package loads nothing; the library is loaded on first use.
"""
