"""GB300-native N-2 contingency screening with a probabilistic Risk Index.

The compute path lives in the CUDA library ``libcs`` (``csrc/``), reached
through the thin ctypes binding :mod:`paper_2512_08465_gb300.cs`.  Importing the
package does not load the library; ``cs`` does, and fails loudly when it is
missing.  :mod:`paper_2512_08465_gb300.synth` draws the seeded synthetic
networks used by tests and benchmarks.
"""
__all__ = ["synth", "cs"]
__version__ = "0.1.0"
