"""GB300-native IMPM elastomer substep (arXiv 2405.02914, Sec. III-A).

``paper_2405_02914_gb300.tsim`` is the Python binding of the C-ABI library
``libtsim.so`` (hand-written sm_103a CUDA); ``paper_2405_02914_gb300.inputs``
draws seeded synthetic scenes.  Importing the package itself loads nothing.
"""
