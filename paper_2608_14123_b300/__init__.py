"""dgfas: B300-native FAS multigrid hot path for SIP DG-SEM elliptic problems."""
