"""GB300 (sm_103a) implementation of the subset-gradient path of RDP-regularised PET
reconstruction with preconditioned SGD / SAGA / SVRG.

The C ABI is declared in ``include/pet_gb300.h``; ``paper_2506_04976_gb300.binding`` is
its ctypes binding and fails loudly at import when the compiled library is missing.
``synth`` generates seeded synthetic inputs.
"""
