"""B300-native aprod / LSQR for the Gaia AVU-GSR system (arXiv 2503.22863).

Submodules:
  gsr    - Python binding over the C-ABI library ``libgsr.so`` (the product path)
  synth  - seeded synthetic systems shaped like the paper's workloads
"""
