"""GB300-native fugacity-based multicomponent lattice Boltzmann (arXiv 2306.10652).

The compute path is the C-ABI library ``liblbmfug.so`` (CUDA, sm_103a); the
Python binding in ``lbmfug.py`` only marshals arguments.  Importing this
package loads nothing; ``paper_2306_10652_gb300.lbmfug`` loads the library
and raises if it is missing.
"""
