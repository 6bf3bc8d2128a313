"""GB300-native guiding-centre transport of solar energetic electrons (arXiv:2403.06706).

The compute path is the C-ABI library ``libgcpush.so`` (hand-written CUDA for
sm_103a, sources in ``csrc/``), reached through the thin ctypes binding in
``gcpush``. ``synth`` builds the seeded synthetic inputs.
"""
__all__ = ["synth", "gcpush"]
