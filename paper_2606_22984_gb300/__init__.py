"""GB300-native FlashVAN hot path: batched ancestral sampling, teacher-forced
log q, Ising energies, free energies, REINFORCE backward and neural MH, all in
hand-written sm_103a CUDA behind the C-ABI library ``libsg`` (``include/sg.h``).

Importing this package does not load the CUDA library; the first call into
``paper_2606_22984_gb300.sg`` does, and raises if it is missing.
"""
