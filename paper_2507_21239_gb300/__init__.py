"""GB300-native representative-particle dust coagulation (mcdust hot path).

Importing the package loads nothing: the CUDA library is loaded by
``paper_2507_21239_gb300.mcd`` on first use.
"""
