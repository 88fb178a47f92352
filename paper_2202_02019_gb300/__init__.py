"""CD-CCSD vvvv ladder on GB300 (sm_103a): C-ABI library + thin binding."""
