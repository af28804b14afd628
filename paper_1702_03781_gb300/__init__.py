"""GB300-native HARP fill and MBF solve for large irregular antenna arrays.

Importing the package loads nothing compiled; `paper_1702_03781_gb300.harp`
loads the CUDA library (and fails loudly when it is missing).
"""
__all__ = ["synth"]
