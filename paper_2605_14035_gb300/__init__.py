"""GB300-native isoparametric finite-element assembly (P1/P2, curves, surfaces, bulk)."""
